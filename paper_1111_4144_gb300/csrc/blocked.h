// Blocked large-order path (blocked.cu), called by api.cu.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/cholinv.h"

namespace cholinv {

// Device workspace of one blocked call (matrices are processed one at a time).
size_t blocked_workspace_bytes(int dtype, int n, int refine);

// Factor (and, if want_inv, invert) `batch` dense n x n matrices stored back
// to back.  X is the working storage and receives the full Hermitian
// inverse; R (optional) receives the factor.  Complex matrices go through
// their real symmetric embedding of order 2n (the inverse only, R NULL).
// tc: 0 CUDA-core products; 1 tensor-core TF32; 2 tensor-core TF32 with the
// three-product split (FP32-level accuracy).  refine_steps (FP32): steps of
// X <- X + X (I - A X), the residual in compensated FP32 pairs, or in FP64
// with resid64.  err_word receives CHOL_ERR_TIMEOUT if a tensor-core kernel
// gave up waiting.
chol_status_t blocked_run(int dtype, int32_t batch, int32_t n, const void* A, void* R, void* X, int32_t* info,
                          int pivot64, int refine_steps, int resid64, int want_inv, int tc, int* err_word, void* ws,
                          cudaStream_t s);

// Kernel timing (chol_blocked_timing): kinds of recorded products.
constexpr int kBlkTrailingUpdate = 0;  // A_>K,>K -= R_K,>K^T R_K,>K (tensor cores)
constexpr int kBlkInverseProduct = 1;  // P = R_I,>I X_>I,>I (tensor cores)
constexpr int kBlkResidual = 2;        // refinement: E = I - A X (FP64 accumulation)
constexpr int kBlkCorrection = 3;      // refinement: X E
constexpr int kBlkWholeCall = 4;       // one matrix's whole factor + inverse (+ refinement)
constexpr int kBlkTimingKinds = 5;
void blocked_timing_enable(int on);
cudaError_t blocked_timing_read(int kind, float* ms, double* flops, int* launches);

}  // namespace cholinv
