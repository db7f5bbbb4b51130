// Batched kernels instantiated for one element type (double).
#include "launch.cuh"

namespace cholinv {

cudaError_t launch_class_f64(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    return launch_class<double>(p, cls, upper, s, dry);
}

}  // namespace cholinv
