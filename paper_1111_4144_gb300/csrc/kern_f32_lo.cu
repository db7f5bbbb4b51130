// Batched kernels for element type float, matrix orders 1..14.
#include "launch.cuh"

namespace cholinv {

cudaError_t launch_class_f32_lo(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    return launch_class_half<float, true>(p, cls, upper, s, dry);
}

int class_variants_f32_lo(int cls) { return class_variants_half<float, true>(cls); }

}  // namespace cholinv
