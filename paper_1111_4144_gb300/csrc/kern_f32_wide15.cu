// Wide kernels (one warp per matrix, registers) for FP32 orders 63 and 64.
#include "wide.cuh"

namespace cholinv {

cudaError_t launch_wide_f32_15(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    return launch_wide_range<63, 64>(p, cls, upper, s, dry);
}

}  // namespace cholinv
