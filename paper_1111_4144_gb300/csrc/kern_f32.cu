// Batched kernels instantiated for one element type (float).
#include "launch.cuh"

namespace cholinv {

cudaError_t launch_class_f32(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    return launch_class<float>(p, cls, upper, s, dry);
}

}  // namespace cholinv
