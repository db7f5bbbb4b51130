// Wide kernels (one warp per matrix, registers) for FP32 orders 53 and 54.
#include "wide.cuh"

namespace cholinv {

cudaError_t launch_wide_f32_10(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    return launch_wide_range<53, 54>(p, cls, upper, s, dry);
}

}  // namespace cholinv
