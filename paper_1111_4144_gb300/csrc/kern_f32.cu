// Batched kernels instantiated for one element type (float).
#include "launch.cuh"

namespace cholinv {

cudaError_t launch_batched_f32(const BatchParams& p, cudaStream_t s, bool dry) {
    return launch_batched<float>(p, s, dry);
}

}  // namespace cholinv
