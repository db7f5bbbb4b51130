// Wide kernels (one warp per matrix, registers) for FP32 orders 59 and 60.
#include "wide.cuh"

namespace cholinv {

cudaError_t launch_wide_f32_13(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    return launch_wide_range<59, 60>(p, cls, upper, s, dry);
}

}  // namespace cholinv
