// Size-class dispatch across the per-type, per-half translation units.
#include "batched.cuh"
#include "dispatch.h"

namespace cholinv {

constexpr int kSplit = 14;  // must match kSplitN in launch.cuh

cudaError_t launch_class_f32_lo(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
cudaError_t launch_class_f32_hi(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
int class_variants_f32_lo(int cls);
int class_variants_f32_hi(int cls);

cudaError_t launch_class_f32(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    return cls <= kSplit ? launch_class_f32_lo(p, cls, upper, s, dry) : launch_class_f32_hi(p, cls, upper, s, dry);
}

int class_variants_f32(int cls) { return cls <= kSplit ? class_variants_f32_lo(cls) : class_variants_f32_hi(cls); }

cudaError_t launch_wide_f32_0(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
cudaError_t launch_wide_f32_1(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
cudaError_t launch_wide_f32_2(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
cudaError_t launch_wide_f32_3(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
cudaError_t launch_wide_f32_4(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
cudaError_t launch_wide_f32_5(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
cudaError_t launch_wide_f32_6(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
cudaError_t launch_wide_f32_7(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);

// orders 33..64, four per translation unit
cudaError_t launch_wide_f32(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    switch ((cls - 33) / 4) {
        case 0: return launch_wide_f32_0(p, cls, upper, s, dry);
        case 1: return launch_wide_f32_1(p, cls, upper, s, dry);
        case 2: return launch_wide_f32_2(p, cls, upper, s, dry);
        case 3: return launch_wide_f32_3(p, cls, upper, s, dry);
        case 4: return launch_wide_f32_4(p, cls, upper, s, dry);
        case 5: return launch_wide_f32_5(p, cls, upper, s, dry);
        case 6: return launch_wide_f32_6(p, cls, upper, s, dry);
        case 7: return launch_wide_f32_7(p, cls, upper, s, dry);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_class_f64_lo(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
cudaError_t launch_class_f64_hi(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
int class_variants_f64_lo(int cls);
int class_variants_f64_hi(int cls);

cudaError_t launch_class_f64(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    return cls <= kSplit ? launch_class_f64_lo(p, cls, upper, s, dry) : launch_class_f64_hi(p, cls, upper, s, dry);
}

int class_variants_f64(int cls) { return cls <= kSplit ? class_variants_f64_lo(cls) : class_variants_f64_hi(cls); }

cudaError_t launch_class_c64_lo(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
cudaError_t launch_class_c64_hi(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
int class_variants_c64_lo(int cls);
int class_variants_c64_hi(int cls);

cudaError_t launch_class_c64(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    return cls <= kSplit ? launch_class_c64_lo(p, cls, upper, s, dry) : launch_class_c64_hi(p, cls, upper, s, dry);
}

int class_variants_c64(int cls) { return cls <= kSplit ? class_variants_c64_lo(cls) : class_variants_c64_hi(cls); }

cudaError_t launch_class_c128_lo(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
cudaError_t launch_class_c128_hi(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
int class_variants_c128_lo(int cls);
int class_variants_c128_hi(int cls);

cudaError_t launch_class_c128(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    return cls <= kSplit ? launch_class_c128_lo(p, cls, upper, s, dry) : launch_class_c128_hi(p, cls, upper, s, dry);
}

int class_variants_c128(int cls) { return cls <= kSplit ? class_variants_c128_lo(cls) : class_variants_c128_hi(cls); }

}  // namespace cholinv
