// Batched kernels for element type complex float, matrix orders 30..32 and the orders above 32.
#include "launch.cuh"

namespace cholinv {

cudaError_t launch_class_c64_r4(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    return launch_class_range<cpx<float>, 30, 32>(p, cls, upper, s, dry);
}

int class_variants_c64_r4(int cls) { return class_variants_range<cpx<float>, 30, 32>(cls); }

}  // namespace cholinv
