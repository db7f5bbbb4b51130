// Batched kernels for element type double, matrix orders 15..20.
#include "launch.cuh"

namespace cholinv {

cudaError_t launch_class_f64_r1(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    return launch_class_range<double, 15, 20>(p, cls, upper, s, dry);
}

int class_variants_f64_r1(int cls) { return class_variants_range<double, 15, 20>(cls); }

}  // namespace cholinv
