// Batched kernels instantiated for one element type (cpx<double>).
#include "launch.cuh"

namespace cholinv {

cudaError_t launch_class_c128(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    return launch_class<cpx<double>>(p, cls, upper, s, dry);
}

}  // namespace cholinv
