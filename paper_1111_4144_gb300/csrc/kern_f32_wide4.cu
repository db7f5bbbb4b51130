// Wide kernels (one warp per matrix, registers) for FP32 orders 41 and 42.
#include "wide.cuh"

namespace cholinv {

cudaError_t launch_wide_f32_4(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    return launch_wide_range<41, 42>(p, cls, upper, s, dry);
}

}  // namespace cholinv
