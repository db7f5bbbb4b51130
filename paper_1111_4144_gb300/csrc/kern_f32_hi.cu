// Batched kernels for element type float, matrix orders 15..64.
#include "launch.cuh"

namespace cholinv {

cudaError_t launch_class_f32_hi(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    return launch_class_half<float, false>(p, cls, upper, s, dry);
}

int class_variants_f32_hi(int cls) { return class_variants_half<float, false>(cls); }

}  // namespace cholinv
