// Batched kernels instantiated for one element type (cpx<double>).
#include "launch.cuh"

namespace cholinv {

cudaError_t launch_batched_c128(const BatchParams& p, cudaStream_t s, bool dry) {
    return launch_batched<cpx<double>>(p, s, dry);
}

}  // namespace cholinv
