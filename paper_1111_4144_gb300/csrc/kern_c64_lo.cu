// Batched kernels for element type cpx<float>, matrix orders 1..14.
#include "launch.cuh"

namespace cholinv {

cudaError_t launch_class_c64_lo(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    return launch_class_half<cpx<float>, true>(p, cls, upper, s, dry);
}

int class_variants_c64_lo(int cls) { return class_variants_half<cpx<float>, true>(cls); }

}  // namespace cholinv
