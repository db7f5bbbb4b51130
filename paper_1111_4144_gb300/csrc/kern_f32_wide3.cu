// Wide kernels (one warp per matrix, registers) for FP32 orders 39 and 40.
#include "wide.cuh"

namespace cholinv {

cudaError_t launch_wide_f32_3(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    return launch_wide_range<39, 40>(p, cls, upper, s, dry);
}

}  // namespace cholinv
