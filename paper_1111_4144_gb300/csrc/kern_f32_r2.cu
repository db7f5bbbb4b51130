// Batched kernels for element type float, matrix orders 21..25.
#include "launch.cuh"

namespace cholinv {

cudaError_t launch_class_f32_r2(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    return launch_class_range<float, 21, 25>(p, cls, upper, s, dry);
}

int class_variants_f32_r2(int cls) { return class_variants_range<float, 21, 25>(cls); }

}  // namespace cholinv
