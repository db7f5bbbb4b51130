// Batched kernels for element type double, matrix orders 1..14.
#include "launch.cuh"

namespace cholinv {

cudaError_t launch_class_f64_lo(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    return launch_class_half<double, true>(p, cls, upper, s, dry);
}

int class_variants_f64_lo(int cls) { return class_variants_half<double, true>(cls); }

}  // namespace cholinv
