// Wide kernels (one warp per matrix, registers) for FP32 orders 37 and 38.
#include "wide.cuh"

namespace cholinv {

cudaError_t launch_wide_f32_2(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    return launch_wide_range<37, 38>(p, cls, upper, s, dry);
}

}  // namespace cholinv
