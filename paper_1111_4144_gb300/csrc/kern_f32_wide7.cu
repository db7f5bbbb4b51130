// Wide kernels (one warp per matrix, registers) for FP32 orders 47 and 48.
#include "wide.cuh"

namespace cholinv {

cudaError_t launch_wide_f32_7(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    return launch_wide_range<47, 48>(p, cls, upper, s, dry);
}

}  // namespace cholinv
