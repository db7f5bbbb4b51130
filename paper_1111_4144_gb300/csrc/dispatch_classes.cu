// Size-class dispatch across the per-type, per-order-range translation units.
#include "batched.cuh"
#include "dispatch.h"

namespace cholinv {

// the order ranges of the kern_<type>_r<k>.cu translation units (launch.cuh)
static int class_range(int cls) { return cls <= 14 ? 0 : cls <= 20 ? 1 : cls <= 25 ? 2 : cls <= 29 ? 3 : 4; }

cudaError_t launch_class_f32_r0(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
int class_variants_f32_r0(int cls);
cudaError_t launch_class_f32_r1(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
int class_variants_f32_r1(int cls);
cudaError_t launch_class_f32_r2(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
int class_variants_f32_r2(int cls);
cudaError_t launch_class_f32_r3(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
int class_variants_f32_r3(int cls);
cudaError_t launch_class_f32_r4(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
int class_variants_f32_r4(int cls);

cudaError_t launch_class_f32(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    switch (class_range(cls)) {
        case 0: return launch_class_f32_r0(p, cls, upper, s, dry);
        case 1: return launch_class_f32_r1(p, cls, upper, s, dry);
        case 2: return launch_class_f32_r2(p, cls, upper, s, dry);
        case 3: return launch_class_f32_r3(p, cls, upper, s, dry);
        case 4: return launch_class_f32_r4(p, cls, upper, s, dry);
    }
    return cudaErrorInvalidValue;
}

int class_variants_f32(int cls) {
    switch (class_range(cls)) {
        case 0: return class_variants_f32_r0(cls);
        case 1: return class_variants_f32_r1(cls);
        case 2: return class_variants_f32_r2(cls);
        case 3: return class_variants_f32_r3(cls);
        case 4: return class_variants_f32_r4(cls);
    }
    return 1;
}

cudaError_t launch_class_f64_r0(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
int class_variants_f64_r0(int cls);
cudaError_t launch_class_f64_r1(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
int class_variants_f64_r1(int cls);
cudaError_t launch_class_f64_r2(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
int class_variants_f64_r2(int cls);
cudaError_t launch_class_f64_r3(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
int class_variants_f64_r3(int cls);
cudaError_t launch_class_f64_r4(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
int class_variants_f64_r4(int cls);

cudaError_t launch_class_f64(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    switch (class_range(cls)) {
        case 0: return launch_class_f64_r0(p, cls, upper, s, dry);
        case 1: return launch_class_f64_r1(p, cls, upper, s, dry);
        case 2: return launch_class_f64_r2(p, cls, upper, s, dry);
        case 3: return launch_class_f64_r3(p, cls, upper, s, dry);
        case 4: return launch_class_f64_r4(p, cls, upper, s, dry);
    }
    return cudaErrorInvalidValue;
}

int class_variants_f64(int cls) {
    switch (class_range(cls)) {
        case 0: return class_variants_f64_r0(cls);
        case 1: return class_variants_f64_r1(cls);
        case 2: return class_variants_f64_r2(cls);
        case 3: return class_variants_f64_r3(cls);
        case 4: return class_variants_f64_r4(cls);
    }
    return 1;
}

cudaError_t launch_class_c64_r0(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
int class_variants_c64_r0(int cls);
cudaError_t launch_class_c64_r1(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
int class_variants_c64_r1(int cls);
cudaError_t launch_class_c64_r2(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
int class_variants_c64_r2(int cls);
cudaError_t launch_class_c64_r3(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
int class_variants_c64_r3(int cls);
cudaError_t launch_class_c64_r4(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
int class_variants_c64_r4(int cls);

cudaError_t launch_class_c64(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    switch (class_range(cls)) {
        case 0: return launch_class_c64_r0(p, cls, upper, s, dry);
        case 1: return launch_class_c64_r1(p, cls, upper, s, dry);
        case 2: return launch_class_c64_r2(p, cls, upper, s, dry);
        case 3: return launch_class_c64_r3(p, cls, upper, s, dry);
        case 4: return launch_class_c64_r4(p, cls, upper, s, dry);
    }
    return cudaErrorInvalidValue;
}

int class_variants_c64(int cls) {
    switch (class_range(cls)) {
        case 0: return class_variants_c64_r0(cls);
        case 1: return class_variants_c64_r1(cls);
        case 2: return class_variants_c64_r2(cls);
        case 3: return class_variants_c64_r3(cls);
        case 4: return class_variants_c64_r4(cls);
    }
    return 1;
}

cudaError_t launch_class_c128_r0(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
int class_variants_c128_r0(int cls);
cudaError_t launch_class_c128_r1(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
int class_variants_c128_r1(int cls);
cudaError_t launch_class_c128_r2(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
int class_variants_c128_r2(int cls);
cudaError_t launch_class_c128_r3(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
int class_variants_c128_r3(int cls);
cudaError_t launch_class_c128_r4(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
int class_variants_c128_r4(int cls);

cudaError_t launch_class_c128(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    switch (class_range(cls)) {
        case 0: return launch_class_c128_r0(p, cls, upper, s, dry);
        case 1: return launch_class_c128_r1(p, cls, upper, s, dry);
        case 2: return launch_class_c128_r2(p, cls, upper, s, dry);
        case 3: return launch_class_c128_r3(p, cls, upper, s, dry);
        case 4: return launch_class_c128_r4(p, cls, upper, s, dry);
    }
    return cudaErrorInvalidValue;
}

int class_variants_c128(int cls) {
    switch (class_range(cls)) {
        case 0: return class_variants_c128_r0(cls);
        case 1: return class_variants_c128_r1(cls);
        case 2: return class_variants_c128_r2(cls);
        case 3: return class_variants_c128_r3(cls);
        case 4: return class_variants_c128_r4(cls);
    }
    return 1;
}

cudaError_t launch_wide_f32_0(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
cudaError_t launch_wide_f32_1(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
cudaError_t launch_wide_f32_2(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
cudaError_t launch_wide_f32_3(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
cudaError_t launch_wide_f32_4(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
cudaError_t launch_wide_f32_5(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
cudaError_t launch_wide_f32_6(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
cudaError_t launch_wide_f32_7(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
cudaError_t launch_wide_f32_8(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
cudaError_t launch_wide_f32_9(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
cudaError_t launch_wide_f32_10(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
cudaError_t launch_wide_f32_11(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
cudaError_t launch_wide_f32_12(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
cudaError_t launch_wide_f32_13(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
cudaError_t launch_wide_f32_14(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
cudaError_t launch_wide_f32_15(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);

// orders 33..64, two per translation unit
cudaError_t launch_wide_f32(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    switch ((cls - 33) / 2) {
        case 0: return launch_wide_f32_0(p, cls, upper, s, dry);
        case 1: return launch_wide_f32_1(p, cls, upper, s, dry);
        case 2: return launch_wide_f32_2(p, cls, upper, s, dry);
        case 3: return launch_wide_f32_3(p, cls, upper, s, dry);
        case 4: return launch_wide_f32_4(p, cls, upper, s, dry);
        case 5: return launch_wide_f32_5(p, cls, upper, s, dry);
        case 6: return launch_wide_f32_6(p, cls, upper, s, dry);
        case 7: return launch_wide_f32_7(p, cls, upper, s, dry);
        case 8: return launch_wide_f32_8(p, cls, upper, s, dry);
        case 9: return launch_wide_f32_9(p, cls, upper, s, dry);
        case 10: return launch_wide_f32_10(p, cls, upper, s, dry);
        case 11: return launch_wide_f32_11(p, cls, upper, s, dry);
        case 12: return launch_wide_f32_12(p, cls, upper, s, dry);
        case 13: return launch_wide_f32_13(p, cls, upper, s, dry);
        case 14: return launch_wide_f32_14(p, cls, upper, s, dry);
        case 15: return launch_wide_f32_15(p, cls, upper, s, dry);
    }
    return cudaErrorInvalidValue;
}

}  // namespace cholinv
