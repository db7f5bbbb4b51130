// Entry points of the per-dtype translation units, called by api.cu.
#pragma once

#include <cuda_runtime.h>

namespace cholinv {

struct BatchParams;
struct BwdParams;
struct MmseParams;

struct DeviceInfo {
    int sms = 0;
};
DeviceInfo device_info();  // defined in api.cu

// Launch the kernel of size class `cls` (matrices of order cls; at most
// `upper` of them) on stream s.  dry = true only performs the kernel's
// one-time set-up (before a stream capture) and launches nothing.
cudaError_t launch_class_f32(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
cudaError_t launch_class_f64(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
cudaError_t launch_class_c64(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
cudaError_t launch_class_c128(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);

// FP32 orders 33..64 on the register-resident wide kernel (kern_f32_wide*.cu).
cudaError_t launch_wide_f32(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);

// Number of kernel variants of an order (for the autotuner).
int class_variants_f32(int cls);
int class_variants_f64(int cls);
int class_variants_c64(int cls);
int class_variants_c128(int cls);

// The tuning table (tune.cu): the variant to launch for (dtype, order); 0 by default.
int variant_of(int dtype, int order);

// Refinement pass (refine.cu): FP32 / complex64 only.  steps Newton-Schulz
// steps on every matrix, or (automatic) one step where max_i a_ii x_ii > 4096.
cudaError_t launch_refine(int dtype, const BatchParams& p, int steps, int automatic, cudaStream_t s, bool dry);

// FP64-pivot pass of CHOL_FLAG_PIVOT64_AUTO (refine.cu): redoes the matrices
// whose info the FP32 pass set to kInfoRedo; a no-op for FP64 value types.
cudaError_t launch_redo(int dtype, const BatchParams& p, cudaStream_t s, bool dry);

// MMSE filters (mmse.cu): stage 0 forms A = H^* H + s2 I, stage 1 W = X H^*.
cudaError_t launch_mmse(int dtype, int stage, const MmseParams& p, double s2, cudaStream_t s, bool dry);

// The whole batch in one persistent launch of the warp body (refine.cu;
// CHOL_FLAG_SINGLE_LAUNCH); *work must be zero.
cudaError_t launch_single(int dtype, const BatchParams& p, int* work, cudaStream_t s, bool dry);

// Adjoint dA = -X (G + G^H)/2 X (adjoint.cu).
cudaError_t launch_backward(int dtype, const BwdParams& p, cudaStream_t s, bool dry);

}  // namespace cholinv
