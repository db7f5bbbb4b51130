// Wide kernels (one warp per matrix, registers) for FP32 orders 35 and 36.
#include "wide.cuh"

namespace cholinv {

cudaError_t launch_wide_f32_1(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    return launch_wide_range<35, 36>(p, cls, upper, s, dry);
}

}  // namespace cholinv
