// Wide kernels (one warp per matrix, registers) for FP32 orders 45 and 46.
#include "wide.cuh"

namespace cholinv {

cudaError_t launch_wide_f32_6(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    return launch_wide_range<45, 46>(p, cls, upper, s, dry);
}

}  // namespace cholinv
