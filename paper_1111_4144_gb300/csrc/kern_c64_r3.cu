// Batched kernels for element type complex float, matrix orders 26..29.
#include "launch.cuh"

namespace cholinv {

cudaError_t launch_class_c64_r3(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    return launch_class_range<cpx<float>, 26, 29>(p, cls, upper, s, dry);
}

int class_variants_c64_r3(int cls) { return class_variants_range<cpx<float>, 26, 29>(cls); }

}  // namespace cholinv
