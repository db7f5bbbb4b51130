// Wide kernels (one warp per matrix, registers) for FP32 orders 33 and 34.
#include "wide.cuh"

namespace cholinv {

cudaError_t launch_wide_f32_0(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    return launch_wide_range<33, 34>(p, cls, upper, s, dry);
}

}  // namespace cholinv
