// Wide kernels (one warp per matrix, registers) for FP32 orders 61 and 62.
#include "wide.cuh"

namespace cholinv {

cudaError_t launch_wide_f32_14(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    return launch_wide_range<61, 62>(p, cls, upper, s, dry);
}

}  // namespace cholinv
