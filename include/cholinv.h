/*
 * cholinv — batched Cholesky factorisation and direct inversion of Hermitian
 * positive-definite matrices on GB300 (sm_103a).
 *
 * Method: Krishnamoorthy & Menon, "Matrix Inversion Using Cholesky
 * Decomposition" (arXiv 1111.4144).
 *   - Factor (Sec. II, Eqs. 2-4): A = R^* R, R upper triangular with a real,
 *     positive diagonal, computed row by row:
 *       r_ii = sqrt(a_ii - sum_{k<i} r_ki^* r_ki)                      (Eq. 3)
 *       r_ij = (a_ij - sum_{k<i} r_ki^* r_kj) / r_ii,  j > i           (Eq. 4)
 *   - Inverse (Sec. IV.A, Eqs. 20-24): X = A^{-1} from R X = S, where
 *     S = diag(1/r_ii) is the known upper part of B = R^{-*}; only x_ij with
 *     i <= j are solved, rows from the last to the first:
 *       x_ij = (s_ij - sum_{k>i} r_ik x~_kj) / r_ii,
 *       x~_kj = x_kj (k <= j), conj(x_jk) (k > j).
 *     No R^{-1} and no B is formed.
 *
 * Conventions shared by every call
 *   Pointers.  Every array argument is a DEVICE pointer (cudaMalloc'd or
 *     managed).  The caller owns every buffer; the library keeps no pointer
 *     after a call returns (except inside a plan, see chol_plan_*).  The
 *     batched calls allocate nothing.
 *   Stream.  `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *     default stream).  Calls only enqueue work and never synchronise, so
 *     they may be captured into a CUDA graph; errors found on the device are
 *     reported through `info` and chol_last_device_error().  A batched call
 *     that launches kernels for 8 or more orders forks them onto side streams
 *     and joins them back into `stream` before it returns (within a capture:
 *     parallel branches of the graph).  The side streams (8 non-blocking
 *     streams and 9 events per host thread and device) are created by the
 *     first such call made outside a capture and kept until the process
 *     ends; a call inside a capture before they exist runs its orders in
 *     sequence on `stream`.
 *   Element types.  CHOL_F32 float, CHOL_F64 double, CHOL_C64 complex float
 *     (interleaved re, im floats), CHOL_C128 complex double.
 *   Sizes and offsets.  Matrix b has order n[b] and starts at element off[b]
 *     (int64, in elements of the dtype) of A, R, X, G and dA.  n == NULL means
 *     every matrix has order max_n; off == NULL means matrix b starts at
 *     element b * (max_n*max_n) (dense) or b * max_n*(max_n+1)/2 (packed).
 *     max_n is a host int and must be >= every n[b].  n[b] == 0 is an empty
 *     matrix (info 0, nothing written).  n[b] < 0 or n[b] > max_n sets
 *     info[b] = -1 and the device error word (CHOL_ERR_ARG).
 *   Large orders.  max_n <= 64 runs the batched kernels (one matrix per
 *     thread, thread group or warp).  max_n > 64 runs the blocked path
 *     (factor and inverse by b x b blocks, products as tiled GEMMs): uniform
 *     batches only (n == NULL, off == NULL), dense layout, one matrix after
 *     another.  There X is the working storage: its lower half is always
 *     written (the full Hermitian inverse), X may not alias A or R, and
 *     refine_steps = -1 means one step.  Complex matrices (CHOL_C64,
 *     CHOL_C128) run as their real symmetric embedding [[B, -C], [C, B]] of
 *     order 2 max_n (A = B + iC; A^{-1} = P + iQ is read back from the
 *     embedding's inverse [[P, -Q], [Q, P]]), in the precision of their real
 *     part (CHOL_C64 as CHOL_F32, with the same precision modes): the inverse
 *     only (R must be NULL; chol_factor_batched returns
 *     CHOL_ERR_UNSUPPORTED), info being the embedding's failing row (in
 *     1..2 max_n), and about twice the arithmetic of complex products.
 *     Other combinations return CHOL_ERR_UNSUPPORTED.
 *   Layout (opts->layout).  0: dense row-major n*n; only the upper triangle
 *     (i <= j) of A is read (Sec. II: the lower part is never needed).
 *     1: upper triangle packed row by row (row i holds columns i..n-1),
 *     n(n+1)/2 elements.  The imaginary part of a diagonal element is ignored.
 *   Outputs.  R (if not NULL) receives the upper triangle; in the dense
 *     layout its strictly lower part is written as zero.  X receives the
 *     upper half of A^{-1}; in the dense layout its strictly lower part is
 *     left untouched unless opts->fill_lower, which writes x_ji = conj(x_ij)
 *     (Sec. III.A / IV.A: "x_ji = x_ij^*").
 *   Aliasing.  R == A, X == A and X == R are allowed (Sec. II notes the
 *     factor may overwrite A): each matrix is read completely before any of
 *     its outputs is written.  Distinct matrices must not overlap.
 *   info.  Device int32[batch] (may be NULL): 0 = success; i > 0 = the
 *     argument of Eq. 3 at 1-based row i was <= 0 or not finite (A not
 *     positive definite, or not representable); the outputs of that matrix
 *     are then filled with NaN.  -1 = invalid n[b].
 *   Workspace.  Batches with per-matrix sizes (n != NULL) are sorted into
 *     size classes on the device, which needs chol_workspace_bytes() bytes of
 *     device memory at `ws` (256-byte aligned).  Uniform batches need none
 *     (ws may be NULL, ws_bytes 0).  Too small a workspace returns
 *     CHOL_ERR_WORKSPACE before anything is launched.
 *   Errors.  Arguments are validated on the host before any launch; a
 *     negative status means nothing was enqueued.
 */
#ifndef CHOLINV_H
#define CHOLINV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CHOL_F32 = 0,
    CHOL_F64 = 1,
    CHOL_C64 = 2,   /* complex float, interleaved */
    CHOL_C128 = 3   /* complex double, interleaved */
} chol_dtype_t;

typedef enum {
    CHOL_OK = 0,
    CHOL_ERR_ARG = -1,          /* invalid argument (host check) or invalid n[b] (device) */
    CHOL_ERR_CUDA = -2,         /* a CUDA runtime call failed */
    CHOL_ERR_UNSUPPORTED = -3,  /* dtype / precision / size combination not implemented */
    CHOL_ERR_TIMEOUT = -4,      /* a bounded device wait gave up */
    CHOL_ERR_WORKSPACE = -5     /* workspace missing, too small or misaligned */
} chol_status_t;

typedef enum {
    CHOL_PREC_NATIVE = 0,       /* all arithmetic in the dtype's precision */
    CHOL_PREC_FP32_REFINE = 1,  /* F32/C64: FP32 body, then refine_steps Newton-Schulz steps
                                   X <- X + X (I - A X) with the residual accumulated in compensated FP32
                                   pairs, or in FP64 with CHOL_FLAG_RESIDUAL_FP64 */
    CHOL_PREC_TF32_REFINE = 2,  /* blocked large-N path (F32): the trailing updates and the inverse-assembly
                                   products on tcgen05 tensor cores as error-corrected TF32 (three TF32
                                   products per FP32 product, FP32-level accuracy), then refine_steps
                                   refinement steps as for CHOL_PREC_FP32_REFINE */
    CHOL_PREC_BF16_REFINE = 3   /* reserved, every call returns CHOL_ERR_UNSUPPORTED: BF16 products (8
                                   significant bits) leave the unrefined inverse of a kappa = 1e4 matrix
                                   without a correct digit, so refinement from it does not converge */
} chol_prec_t;

/* opts->flags */
#define CHOL_FLAG_PIVOT64 0x1     /* F32/C64: accumulate Eq. 3 (the pivot) in FP64 and take its sqrt in FP64 */
#define CHOL_FLAG_GRAD_UPPER 0x2  /* chol_inv_backward: gradient with respect to the upper triangle taken as
                                     the independent parameters (see chol_inv_backward) */
#define CHOL_FLAG_PLAN_TIMING 0x4 /* chol_plan_inv_create only: record timing events around each size-class
                                     kernel (see chol_plan_kernel_ms) */
#define CHOL_FLAG_TF32_SINGLE 0x8 /* CHOL_PREC_TF32_REFINE: single-pass TF32 products (11 significant bits)
                                     instead of the three-product split; only for kappa * 2^-11 << 1 */
#define CHOL_FLAG_LDL 0x20         /* the LDL form (Sec. II.A, Eqs. 9-11; Sec. IV.B, Eqs. 25-29): A = R^* D R with R
                                     unit upper and D = diag(d_i), no square roots; X as for Cholesky.  R, when
                                     written, holds d_i on its diagonal (the unit diagonal is implied).  Batched
                                     path only (orders <= 64: up to 32 on the same thread-per-matrix and
                                     group kernels as the Cholesky form, above on the one-matrix-per-warp
                                     kernel); not with CHOL_FLAG_PIVOT64 */
#define CHOL_FLAG_PIVOT64_AUTO 0x40 /* F32/C64 batched calls: FP64 pivots only for the matrices that need them.
                                     The FP32 pass watches Eq. 3 at every row i; a matrix whose argument
                                     t_i falls below 2^-10 a_ii (cancellation: about 10 of FP32's 24 bits
                                     lost), or is <= 0 or not finite, is not stored by that pass and is
                                     factored and inverted again with the sum of Eq. 3 accumulated in FP64
                                     (as CHOL_FLAG_PIVOT64), in a second kernel over the batch.  Since
                                     t_i >= lambda_min and a_ii <= lambda_max, a matrix with kappa_2 < 2^10
                                     is never redone.  info must not be NULL (CHOL_ERR_ARG): it carries the
                                     list of matrices to redo between the two kernels.  The number redone
                                     is counted on the device (chol_pivot64_redo_count).  FP64 value types
                                     ignore the flag; the blocked path (max_n > 64) takes it as
                                     CHOL_FLAG_PIVOT64.  Not with CHOL_FLAG_LDL */
#define CHOL_FLAG_RESIDUAL_FP64 0x80 /* refinement (CHOL_PREC_FP32_REFINE / CHOL_PREC_TF32_REFINE): accumulate the
                                     residual I - A X in IEEE FP64.  Without it the residual's sums run in
                                     compensated FP32 pairs (Ogita-Rump-Oishi Dot2: exact products, error-free
                                     sums, about 48 significant bits) and no FP64 arithmetic is used; GPUs
                                     whose FP64 rate is a small fraction of FP32's run that several times
                                     faster */
#define CHOL_FLAG_METHOD_ES 0x100  /* batched path, for comparison: the upper half of X by the existing method
                                     "Equation Solving" (Sec. III.A, Eq. 15) instead of the proposed one: for
                                     each column j the forward solve R^* b = e_j, then the back substitution
                                     R x_j = b for x_ij, i <= j.  Same results as the proposed method (its
                                     b_i, i <= j, are the s_ij of Eq. 24); the forward solves are its extra
                                     work.  One matrix per warp; not with CHOL_FLAG_LDL */
#define CHOL_FLAG_METHOD_TMO 0x200 /* batched path, for comparison: the existing method "Triangular Matrix
                                     Operations" (Sec. III.B, Eqs. 16-19): M = R^{-1} from R m_i = e_i, then
                                     the upper half of X = M M^*.  One matrix per warp; not with
                                     CHOL_FLAG_LDL or CHOL_FLAG_METHOD_ES */
#define CHOL_FLAG_SINGLE_LAUNCH 0x400 /* batched path: one persistent kernel for the whole batch instead of one
                                     kernel per order.  Its warps take the matrices one at a time from a
                                     device counter, largest orders first (after the bucketing of a batch
                                     with per-matrix sizes), and run the one-matrix-per-warp form at each
                                     matrix's own order, so an eager call launches no kernel for an order
                                     that is absent.  The per-order kernels are faster where each order has
                                     many matrices; this form is the comparison, and the choice for batches
                                     spread thin over many orders.  Calls with this flag on a uniform batch
                                     (n == NULL) share a per-device counter: serialise them */
#define CHOL_FLAG_PLAN_ORDERS 0x10 /* chol_plan_inv_create only, batches with per-matrix sizes: read n once
                                     at creation (synchronously) and record kernels only for the orders
                                     present then, instead of one per order 1..max_n.  At every replay a
                                     matrix whose order was not present at creation is not inverted: its
                                     info is -1 and the device error word becomes CHOL_ERR_ARG */

typedef struct {
    int32_t prec;          /* chol_prec_t */
    int32_t refine_steps;  /* CHOL_PREC_FP32_REFINE: 0, 1 or 2; -1 = automatic (see chol_inv_batched) */
    int32_t fill_lower;    /* dense layout: also write the strictly lower half of X */
    int32_t layout;        /* 0 dense row-major, 1 packed upper */
    int32_t flags;         /* CHOL_FLAG_* */
    int32_t reserved;      /* must be 0 */
    uint64_t orders;       /* batches with per-matrix sizes (n != NULL, max_n <= 64): the orders that may
                              occur, bit c-1 for order c; 0 = any order 1..max_n.  A call launches a
                              size-class kernel for each order of the set only (an eager call cannot
                              read n on the host without synchronising, so without a set it launches one
                              for every order 1..max_n, the absent ones exiting at once).  A matrix of an
                              order outside the set gets info = -1 and the device error word
                              CHOL_ERR_ARG, as an order outside 0..max_n.  Ignored for uniform batches
                              and the blocked path */
} chol_opts_t;

/* Call identifiers for chol_workspace_bytes(). */
#define CHOL_CALL_FACTOR 0
#define CHOL_CALL_INV 1
#define CHOL_CALL_BACKWARD 2
#define CHOL_CALL_INV_HOST 3
#define CHOL_CALL_MMSE 4

/*
 * chol_factor_batched — Cholesky factor R of each matrix (Sec. II, Eqs. 3-4).
 *   A: input, R: output (may equal A).  opts may be NULL (defaults: native
 *   precision, dense layout).
 */
chol_status_t chol_factor_batched(chol_dtype_t dt, int32_t batch, const int32_t* n, const int64_t* off,
                                  int32_t max_n, const void* A, void* R, int32_t* info,
                                  const chol_opts_t* opts, void* ws, size_t ws_bytes, void* stream);

/*
 * chol_inv_batched — upper half of X = A^{-1} by the proposed method
 * (Sec. II Eqs. 3-4 fused with Sec. IV.A Eqs. 20-24): the factor stays on
 * chip and the recurrence for X runs on it directly.
 *   A: input; R: optional output of the factor (NULL = not written);
 *   X: output.  With opts->prec = CHOL_PREC_FP32_REFINE (F32 / C64) the
 *   result is refined by refine_steps Newton-Schulz steps
 *   X <- X + X (I - A X), the residual formed from exact products of the
 *   FP32 operands and accumulated in compensated FP32 pairs (about 48
 *   bits) or, with CHOL_FLAG_RESIDUAL_FP64, in FP64.  refine_steps = -1 (automatic) refines a
 *   matrix once when gamma = max_i a_ii x_ii > 4096; gamma lies in
 *   [1, (1 + kappa)^2 / (4 kappa)] with kappa = kappa_2(A), so only
 *   matrices with kappa above about 16,382 can be refined.
 *   Refinement reads A again after X is formed, so X == A is rejected
 *   (CHOL_ERR_ARG) when refine_steps != 0.  CHOL_FLAG_PIVOT64 accumulates
 *   the sum of Eq. 3 in FP64 for F32 / C64 (pivots lost to cancellation).
 */
chol_status_t chol_inv_batched(chol_dtype_t dt, int32_t batch, const int32_t* n, const int64_t* off,
                               int32_t max_n, const void* A, void* R, void* X, int32_t* info,
                               const chol_opts_t* opts, void* ws, size_t ws_bytes, void* stream);

/*
 * chol_inv_backward — adjoint of X = A^{-1} on Hermitian matrices:
 *   dA = -X S X,  S = (G + G^H) / 2
 * (not in the paper; it reuses the forward X and does no refactorisation).
 * For every Hermitian perturbation E, dL = Re<dA, E>_F: dA is the gradient
 * on the Hermitian subspace, itself Hermitian.
 *   X: the forward result in opts->layout, at element offsets xoff[b]
 *   (NULL = contiguous); its upper half is read, the lower half is taken as
 *   the conjugate mirror.  G: dense n*n gradient of the loss with respect
 *   to the full X.  dA: dense n*n output.  G and dA use the element offsets
 *   off[b] of a dense batch (off == NULL: b * max_n^2).
 *   With CHOL_FLAG_GRAD_UPPER, dA is instead the gradient with respect to
 *   the entries the forward call reads (the upper triangle, diagonal real
 *   part): 2 dA_ij above the diagonal, Re(dA_ii) on it, 0 below.  This is
 *   what an autograd system that perturbs entries one at a time expects.
 *   dA may not alias X or G.
 */
chol_status_t chol_inv_backward(chol_dtype_t dt, int32_t batch, const int32_t* n, const int64_t* off,
                                const int64_t* xoff, int32_t max_n, const void* X, const void* G, void* dA,
                                const chol_opts_t* opts, void* ws, size_t ws_bytes, void* stream);

/*
 * chol_inv_batched_host — chol_inv_batched for a batch that lives in HOST
 * memory (Sec. II factor + Sec. IV.A inverse, as chol_inv_batched; the
 * paper has no counterpart for the data movement).
 *   A_host, X_host, n_host, off_host, info_host: host pointers.  Page-locked
 *   (pinned) memory gives full copy speed; with pageable memory the copies
 *   are staged by the driver and lose most of the overlap.  Each chunk's
 *   copies start on a 128-byte boundary of host memory (copies from other
 *   addresses run slower on GB300), so the copy in may also read up to 127
 *   bytes of A_host before the chunk's first matrix, never before A_host
 *   itself; X_host is written only where the batch's matrices are.
 *   Batch layout: either n_host == off_host == NULL (every matrix of order
 *   max_n, stored back to back), or both given, with the matrices stored
 *   back to back in index order (off_host[b+1] = off_host[b] + elements of
 *   matrix b; each chunk's span is checked, CHOL_ERR_ARG otherwise).
 *   Orders <= 64.  In dense layout the whole n x n block of every matrix is
 *   written back (fill_lower is implied); in packed layout the triangle.
 *   R is not produced.  opts (precision, refinement, flags) apply as for
 *   chol_inv_batched.
 * The batch is cut into chunks of whole matrices (up to 16 per call, each at
 * least 8192 matrices or the whole batch) that pass through four device
 * slots and four internal streams (copy in, two for the kernels of
 * alternate chunks, copy out), so the copies of one chunk overlap the
 * kernels and copies of the others.  The
 * call returns once everything is enqueued: `stream` waits for all of it,
 * and the host buffers must stay valid and unmodified until then.
 * ws: device workspace of chol_workspace_bytes(CHOL_CALL_INV_HOST, dt,
 * batch, max_n, n_host != NULL, opts) bytes, 256-byte aligned (it holds the
 * whole batch's orders, offsets and info, each copied in one piece, and the
 * four slots).  Concurrent calls on one device serialise their enqueueing.
 */
chol_status_t chol_inv_batched_host(chol_dtype_t dt, int32_t batch, const int32_t* n_host, const int64_t* off_host,
                                    int32_t max_n, const void* A_host, void* X_host, int32_t* info_host,
                                    const chol_opts_t* opts, void* ws, size_t ws_bytes, void* stream);

/*
 * chol_inv_batched_noalloc — chol_inv_batched for callers that cannot
 * allocate device memory.  The paper has no counterpart; this is a
 * deployment variant of the same computation.
 *
 * Some callers cannot hand the library a workspace: code that runs while a
 * global-mode stream capture is open on another thread (cudaMalloc is
 * prohibited then), real-time host paths where an allocation's latency or
 * failure is not acceptable, and plugins whose host application owns and
 * pools all device memory.  This entry point takes the same arguments as
 * chol_inv_batched without ws/ws_bytes and allocates nothing: the
 * size-class bucketing that a batch with per-matrix sizes needs uses a
 * fixed scratch array compiled into the library (1 KiB plus 4 bytes per
 * matrix for CHOL_NOALLOC_MAX_BATCH matrices, about 4 MiB), which every GPU
 * that loads the library holds until the process exits.
 *
 *   - n != NULL and batch > CHOL_NOALLOC_MAX_BATCH returns
 *     CHOL_ERR_WORKSPACE before anything is launched (uniform batches,
 *     n == NULL, need no scratch and have no limit).
 *   - The first call on a device looks up the scratch array's device
 *     address (cudaGetSymbolAddress, with that device current); make that
 *     first call before any stream capture begins.
 *   - Every call shares the one scratch array and the array keeps the last
 *     call's contents (each call clears the counters it needs before use).
 *     Calls whose executions overlap on the GPU (different streams, or
 *     concurrent graph replays) race on it: serialise them.
 *   - Inputs, outputs, info, opts and the stream are the caller's, as for
 *     chol_inv_batched (refinement included: X == A is then rejected with
 *     CHOL_ERR_ARG); no cudaMalloc, cudaFree or allocating library routine
 *     is called.
 */
#define CHOL_NOALLOC_MAX_BATCH 1048576
chol_status_t chol_inv_batched_noalloc(chol_dtype_t dt, int32_t batch, const int32_t* n, const int64_t* off,
                                       int32_t max_n, const void* A, void* R, void* X, int32_t* info,
                                       const chol_opts_t* opts, void* stream);

/*
 * chol_mmse_batched — linear MMSE filters W = (H^* H + sigma2 I)^{-1} H^*
 * of a batch of channel matrices, the usual consumer of the MIMO
 * covariances A = H^* H + sigma2 I.  With sigma2 = 0 and a square H it
 * inverts a non-Hermitian matrix through a Hermitian one (Sec. III.C): for
 * H = D^*, W = (D D^*)^{-1} D and W^* = D^* (D D^*)^{-1} = D^{-1}, the
 * paper's form; for H = D, W = (D^* D)^{-1} D^* = D^{-1} directly.  The Hermitian inverse is the proposed method (Sec. II
 * Eqs. 3-4 and Sec. IV.A, as chol_inv_batched).  Three steps on `stream`:
 * A = H^* H + sigma2 I (packed, in the workspace), X = A^{-1} (the batched
 * kernels), W = X H^*.
 *   H: matrix b is m[b] x n[b] row-major at element hoff[b] (m == NULL:
 *   every m[b] = max_m; hoff == NULL: b * max_m * max_n).  W: n[b] x m[b]
 *   row-major at element woff[b] (woff == NULL: b * max_n * max_m).
 *   n == NULL: every order is max_n (<= 64).  sigma2 >= 0.  opts: precision,
 *   refinement and flags as for chol_inv_batched (layout and fill_lower do
 *   not apply).  info as for chol_inv_batched; W of a failed matrix is NaN.
 *   ws: chol_workspace_bytes(CHOL_CALL_MMSE, dt, batch, max_n, n != NULL,
 *   opts) bytes, 256-byte aligned.  ((max_m + 1) max_n + max_n (max_n + 1))
 *   elements must fit 96 KB (CHOL_ERR_UNSUPPORTED otherwise).
 */
chol_status_t chol_mmse_batched(chol_dtype_t dt, int32_t batch, const int32_t* n, const int32_t* m,
                                const int64_t* hoff, const int64_t* woff, int32_t max_n, int32_t max_m, const void* H,
                                double sigma2, void* W, int32_t* info, const chol_opts_t* opts, void* ws,
                                size_t ws_bytes, void* stream);

/* Bytes of device workspace that a call with these arguments needs (0 = none). */
size_t chol_workspace_bytes(int32_t call, chol_dtype_t dt, int32_t batch, int32_t max_n, int32_t has_sizes,
                            const chol_opts_t* opts);

/* A static, human-readable description of a status code. */
const char* chol_status_string(chol_status_t status);

/* Synchronises `stream`, then reads and clears the device error word of the
 * current device (CHOL_OK if no kernel reported an error). */
chol_status_t chol_last_device_error(void* stream);

/* Synchronises `stream`, then reads and clears the number of matrices that
 * CHOL_FLAG_PIVOT64_AUTO calls on the current device have redone with FP64
 * pivots (Eq. 3) since the last read.  CHOL_ERR_ARG if count is NULL. */
chol_status_t chol_pivot64_redo_count(void* stream, int64_t* count);

/*
 * Autotuning (not in the paper).  Orders up to 32 have more than one
 * compiled kernel variant (one matrix per thread vs. G threads per matrix,
 * or G vs. 2G threads); which is fastest depends on the GPU.
 * chol_autotune times every variant of every order 1..max_n for dtype dt and
 * layout on a synthetic batch of `batch` matrices on `stream` (each timed
 * launch after L2 is overwritten, as for batches streamed from HBM; it
 * allocates twice L2 for that) and keeps the
 * fastest in a per-process table that all later calls use (plans capture
 * the variant current at creation).  It allocates and frees device memory
 * and synchronises the stream, so it is a set-up call, not for the hot path
 * or a stream capture.  cache_path (may be NULL) receives the choices as a
 * small text file keyed by GPU name; chol_tune_load reads such a file back.
 * chol_tune_variants / chol_tune_get / chol_tune_set inspect or pin the
 * table (variant 0 is the compiled-in default).
 */
chol_status_t chol_autotune(chol_dtype_t dt, int32_t max_n, int32_t layout, int32_t batch, const char* cache_path,
                            void* stream);
chol_status_t chol_tune_load(const char* cache_path);
int32_t chol_tune_variants(chol_dtype_t dt, int32_t order);
int32_t chol_tune_get(chol_dtype_t dt, int32_t order);
chol_status_t chol_tune_set(chol_dtype_t dt, int32_t order, int32_t variant);

/*
 * Kernel timing of the blocked path (orders > 64; not in the paper).
 * chol_blocked_timing(1) starts recording on the calling host thread (and
 * clears what was recorded); from then on every blocked call that thread
 * makes records a CUDA event pair, on the call's stream, around each product
 * of these kinds, with the product's algorithmic flops (2 M N K, or the
 * upper part only where only it is formed):
 *   CHOL_BLK_TRAILING_UPDATE  A_>K,>K -= R_K,>K^* R_K,>K  (Eqs. 3-4 in block form)
 *   CHOL_BLK_INVERSE_PRODUCT  R_I,>I X_>I,>I              (Sec. IV.A in block form)
 *   CHOL_BLK_RESIDUAL         E = I - A X                 (refinement)
 *   CHOL_BLK_CORRECTION       X E                         (refinement)
 *   CHOL_BLK_WHOLE_CALL       each matrix's whole call, flops counted as n^3
 * chol_blocked_timing(0) stops and frees the events.  The events cost
 * launch time, so time a call without them for its throughput.
 * chol_blocked_timing_read waits for the recorded events and returns the
 * summed milliseconds, flops and number of products of one kind since
 * recording started; CHOL_ERR_ARG for an unknown kind, NULL outputs or no
 * recording on this thread.
 */
#define CHOL_BLK_TRAILING_UPDATE 0
#define CHOL_BLK_INVERSE_PRODUCT 1
#define CHOL_BLK_RESIDUAL 2
#define CHOL_BLK_CORRECTION 3
#define CHOL_BLK_WHOLE_CALL 4
chol_status_t chol_blocked_timing(int32_t enable);
chol_status_t chol_blocked_timing_read(int32_t kind, float* ms, double* flops, int32_t* launches);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int32_t chol_version(void);

/*
 * Plans: a batched call recorded once into a CUDA graph and replayed.
 *   chol_plan_inv_create records exactly what chol_inv_batched would enqueue
 *   for these arguments (pointers included) by stream capture on an internal
 *   stream, and instantiates the graph.  The caller keeps every buffer alive
 *   until chol_plan_destroy.  chol_plan_launch replays the graph on `stream`.
 */
typedef struct chol_plan chol_plan_t;

chol_status_t chol_plan_inv_create(chol_plan_t** plan, chol_dtype_t dt, int32_t batch, const int32_t* n,
                                   const int64_t* off, int32_t max_n, const void* A, void* R, void* X,
                                   int32_t* info, const chol_opts_t* opts, void* ws, size_t ws_bytes);
chol_status_t chol_plan_launch(chol_plan_t* plan, void* stream);
chol_status_t chol_plan_destroy(chol_plan_t* plan);

/*
 * Duration in milliseconds of the kernel of matrix order `order` in the
 * plan's most recent replay (the plan must have been created with
 * CHOL_FLAG_PLAN_TIMING and the replay's stream synchronised).  The
 * size-class kernels of a batch with per-matrix sizes run one after another
 * on the replay's stream.
 * CHOL_ERR_ARG if the plan records no timing or no kernel of that order.
 */
chol_status_t chol_plan_kernel_ms(chol_plan_t* plan, int32_t order, float* ms);

#ifdef __cplusplus
}
#endif

#endif /* CHOLINV_H */
