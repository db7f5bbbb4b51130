// Batched kernels for element type double, matrix orders 30..32 and the orders above 32.
#include "launch.cuh"

namespace cholinv {

cudaError_t launch_class_f64_r4(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    return launch_class_range<double, 30, 32>(p, cls, upper, s, dry);
}

int class_variants_f64_r4(int cls) { return class_variants_range<double, 30, 32>(cls); }

}  // namespace cholinv
