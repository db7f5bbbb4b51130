// Batched kernels instantiated for one element type (double).
#include "launch.cuh"

namespace cholinv {

cudaError_t launch_batched_f64(const BatchParams& p, cudaStream_t s, bool dry) {
    return launch_batched<double>(p, s, dry);
}

}  // namespace cholinv
