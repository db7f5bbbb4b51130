// Wide kernels (one warp per matrix, registers) for FP32 orders 51 and 52.
#include "wide.cuh"

namespace cholinv {

cudaError_t launch_wide_f32_9(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    return launch_wide_range<51, 52>(p, cls, upper, s, dry);
}

}  // namespace cholinv
