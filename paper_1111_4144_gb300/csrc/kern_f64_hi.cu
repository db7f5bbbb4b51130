// Batched kernels for element type double, matrix orders 15..64.
#include "launch.cuh"

namespace cholinv {

cudaError_t launch_class_f64_hi(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    return launch_class_half<double, false>(p, cls, upper, s, dry);
}

int class_variants_f64_hi(int cls) { return class_variants_half<double, false>(cls); }

}  // namespace cholinv
