// Batched kernels instantiated for one element type (cpx<float>).
#include "launch.cuh"

namespace cholinv {

cudaError_t launch_class_c64(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    return launch_class<cpx<float>>(p, cls, upper, s, dry);
}

}  // namespace cholinv
