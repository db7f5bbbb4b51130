// Wide kernels (one warp per matrix, registers) for FP32 orders 55 and 56.
#include "wide.cuh"

namespace cholinv {

cudaError_t launch_wide_f32_11(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    return launch_wide_range<55, 56>(p, cls, upper, s, dry);
}

}  // namespace cholinv
