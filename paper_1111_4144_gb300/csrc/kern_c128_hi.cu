// Batched kernels for element type cpx<double>, matrix orders 15..64.
#include "launch.cuh"

namespace cholinv {

cudaError_t launch_class_c128_hi(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    return launch_class_half<cpx<double>, false>(p, cls, upper, s, dry);
}

int class_variants_c128_hi(int cls) { return class_variants_half<cpx<double>, false>(cls); }

}  // namespace cholinv
