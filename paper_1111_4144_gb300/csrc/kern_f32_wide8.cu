// Wide kernels (one warp per matrix, registers) for FP32 orders 49 and 50.
#include "wide.cuh"

namespace cholinv {

cudaError_t launch_wide_f32_8(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    return launch_wide_range<49, 50>(p, cls, upper, s, dry);
}

}  // namespace cholinv
