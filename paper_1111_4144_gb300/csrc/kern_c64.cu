// Batched kernels instantiated for one element type (cpx<float>).
#include "launch.cuh"

namespace cholinv {

cudaError_t launch_batched_c64(const BatchParams& p, cudaStream_t s, bool dry) {
    return launch_batched<cpx<float>>(p, s, dry);
}

}  // namespace cholinv
