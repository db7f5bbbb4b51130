// Wide kernels (one warp per matrix, registers) for FP32 orders 57 and 58.
#include "wide.cuh"

namespace cholinv {

cudaError_t launch_wide_f32_12(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    return launch_wide_range<57, 58>(p, cls, upper, s, dry);
}

}  // namespace cholinv
