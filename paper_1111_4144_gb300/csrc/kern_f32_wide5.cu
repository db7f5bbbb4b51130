// Wide kernels (one warp per matrix, registers) for FP32 orders 43 and 44.
#include "wide.cuh"

namespace cholinv {

cudaError_t launch_wide_f32_5(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    return launch_wide_range<43, 44>(p, cls, upper, s, dry);
}

}  // namespace cholinv
