// Batched kernels for element type double, matrix orders 26..29.
#include "launch.cuh"

namespace cholinv {

cudaError_t launch_class_f64_r3(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    return launch_class_range<double, 26, 29>(p, cls, upper, s, dry);
}

int class_variants_f64_r3(int cls) { return class_variants_range<double, 26, 29>(cls); }

}  // namespace cholinv
