// Batched kernels for element type float, matrix orders 15..20.
#include "launch.cuh"

namespace cholinv {

cudaError_t launch_class_f32_r1(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    return launch_class_range<float, 15, 20>(p, cls, upper, s, dry);
}

int class_variants_f32_r1(int cls) { return class_variants_range<float, 15, 20>(cls); }

}  // namespace cholinv
