// Blocked path for large matrices (order > 64): the paper's factorisation
// (Eqs. 3-4) and inverse recurrence (Sec. IV.A) taken block by block.
//
// Factor, right-looking, panel K of b rows:
//   R_KK      = chol(A_KK)                    Eqs. 3-4 on the diagonal block (one CTA)
//   R_K,>K    = R_KK^{-T} A_K,>K              Eq. 4 for the block row (a GEMM with the
//                                            inverted b x b diagonal block)
//   A_>K,>K  -= R_K,>K^T R_K,>K               the k < i terms of Eqs. 3-4 (upper tiles only)
// Inverse, block rows I = last..first (R X = S, S = diag(1/r_ii)):
//   X_I,>I    = -R_II^{-1} (R_I,>I X_>I,>I)   off-diagonal blocks (x_ij = -(1/r_ii) sum_{k>i} r_ik x~_kj)
//   Z         = R_I,>I X_I,>I^T               the k beyond the block part of the diagonal sums
//   X_II      : the recurrence inside the block with s_ij replaced by s_ij - z_ij
// X is kept full (each new block row is mirrored into its block column) so
// that every product reads plain dense operands.  The matrix lives in X
// (dense row-major, in place); A is only read.
//
// The products run through one tiled GEMM (`k_gemm`); the small triangular
// pieces through single-CTA kernels.  Real element types (FP32, FP64).
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "batched.cuh"
#include "blocked.h"
#include "dispatch.h"
#include "umma.cuh"

namespace cholinv {

// ---------------------------------------------------------------------------
// Tiled GEMM:  C = alpha * op(A) op(B) + beta * C   (or, with `partial`, the
// raw product of one K-slice into partial[z]).  op(A) is M x K: A stored
// row-major M x K (TA = false) or K x M (TA = true); op(B) is K x N: stored
// K x N (TB = false) or N x K (TB = true).  upper != 0 computes only the
// entries with row <= col (tiles wholly below the diagonal are skipped).
// 128 x 128 tiles, BK = 8, 256 threads, 8 x 8 outputs per thread.
// ---------------------------------------------------------------------------
constexpr int GB_M = 128, GB_N = 128, GB_K = 8, GB_THREADS = 256;

template <typename Tin, typename Tacc, typename Tout, bool TA, bool TB>
__global__ void __launch_bounds__(GB_THREADS)
k_gemm(int M, int N, int K, Tacc alpha, const Tin* __restrict__ A, int64_t lda, const Tin* __restrict__ B,
       int64_t ldb, Tacc beta, Tout* C, int64_t ldc, int upper, int kchunk, Tacc* partial) {
    __shared__ Tin As[2][GB_K][GB_M + 4];
    __shared__ Tin Bs[2][GB_K][GB_N + 4];
    const int m0 = blockIdx.y * GB_M, n0 = blockIdx.x * GB_N;
    if (upper && m0 > n0 + GB_N - 1) return;
    const int kb = blockIdx.z * kchunk;
    const int ke = min(K, kb + kchunk);
    const int t = threadIdx.x;
    const int tm = (t / 16) * 8, tn = (t % 16) * 8;
    Tacc acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = Tacc(0);

    auto load = [&](int buf, int k0) {
        // 128 x 8 elements of each operand, 4 per thread
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int f = t + r * GB_THREADS;
            int mm, kk;
            if (TA) { kk = f / GB_M; mm = f % GB_M; } else { mm = f / GB_K; kk = f % GB_K; }
            const int gm = m0 + mm, gk = k0 + kk;
            Tin v = Tin(0);
            if (gm < M && gk < ke) v = TA ? A[(int64_t)gk * lda + gm] : A[(int64_t)gm * lda + gk];
            As[buf][kk][mm] = v;
            int nn, k2;
            if (TB) { nn = f / GB_K; k2 = f % GB_K; } else { k2 = f / GB_N; nn = f % GB_N; }
            const int gn = n0 + nn, gk2 = k0 + k2;
            Tin w = Tin(0);
            if (gn < N && gk2 < ke) w = TB ? B[(int64_t)gn * ldb + gk2] : B[(int64_t)gk2 * ldb + gn];
            Bs[buf][k2][nn] = w;
        }
    };
    int buf = 0;
    if (kb < ke) load(0, kb);
    __syncthreads();
    for (int k0 = kb; k0 < ke; k0 += GB_K) {
        if (k0 + GB_K < ke) load(buf ^ 1, k0 + GB_K);
#pragma unroll
        for (int kk = 0; kk < GB_K; ++kk) {
            Tacc a[8], b[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = (Tacc)As[buf][kk][tm + i];
#pragma unroll
            for (int j = 0; j < 8; ++j) b[j] = (Tacc)Bs[buf][kk][tn + j];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
        buf ^= 1;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int gm = m0 + tm + i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int gn = n0 + tn + j;
            if (gn >= N || (upper && gm > gn)) continue;
            if (partial) {
                partial[((int64_t)blockIdx.z * M + gm) * N + gn] = acc[i][j];
            } else {
                Tacc c = alpha * acc[i][j];
                if (beta != Tacc(0)) c = fma(beta, (Tacc)C[(int64_t)gm * ldc + gn], c);
                C[(int64_t)gm * ldc + gn] = (Tout)c;
            }
        }
    }
}

// Refinement residual E = I - A X for n x n FP32 A (full) and X, each entry
// a compensated FP32 dot product (exact products, error-free sums, about 48
// bits) started at delta_ij, rounded to FP32 once at the end; two entries
// of a row per paired FP32 instruction (f2acc2).  The tiling is k_gemm's
// (128 x 128 tiles, 8 x 8 entries per thread).
__global__ void __launch_bounds__(GB_THREADS)
k_resid_f2(int n, const float* __restrict__ A, const float* __restrict__ X, float* E) {
    __shared__ float As[2][GB_K][GB_M + 4];
    __shared__ float Bs[2][GB_K][GB_N + 4];
    const int m0 = blockIdx.y * GB_M, n0 = blockIdx.x * GB_N;
    const int t = threadIdx.x;
    const int tm = (t / 16) * 8, tn = (t % 16) * 8;
    // acc[i][jj] holds entries (tm + i, tn + 2 jj) and (tm + i, tn + 2 jj + 1)
    f2acc2 acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const int gi = m0 + tm + i, gj = n0 + tn + 2 * jj;
            acc[i][jj].s = make_float2(gi == gj ? 1.f : 0.f, gi == gj + 1 ? 1.f : 0.f);
            acc[i][jj].c = make_float2(0.f, 0.f);
        }
    auto load = [&](int buf, int k0) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int f = t + r * GB_THREADS;
            const int mm = f / GB_K, kk = f % GB_K;
            const int gm = m0 + mm, gk = k0 + kk;
            As[buf][kk][mm] = (gm < n && gk < n) ? A[(int64_t)gm * n + gk] : 0.f;
            const int k2 = f / GB_N, nn = f % GB_N;
            const int gn = n0 + nn, gk2 = k0 + k2;
            Bs[buf][k2][nn] = (gn < n && gk2 < n) ? X[(int64_t)gk2 * n + gn] : 0.f;
        }
    };
    int buf = 0;
    load(0, 0);
    __syncthreads();
    for (int k0 = 0; k0 < n; k0 += GB_K) {
        if (k0 + GB_K < n) load(buf ^ 1, k0 + GB_K);
#pragma unroll
        for (int kk = 0; kk < GB_K; ++kk) {
            float2 a[8], b[4];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float v = -As[buf][kk][tm + i];
                a[i] = make_float2(v, v);
            }
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) b[jj] = make_float2(Bs[buf][kk][tn + 2 * jj], Bs[buf][kk][tn + 2 * jj + 1]);
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) f2_fma2(acc[i][jj], a[i], b[jj]);
        }
        __syncthreads();
        buf ^= 1;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int gm = m0 + tm + i;
        if (gm >= n) continue;
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const int gn = n0 + tn + 2 * jj;
            if (gn < n) E[(int64_t)gm * n + gn] = __fadd_rn(acc[i][jj].s.x, acc[i][jj].c.x);
            if (gn + 1 < n) E[(int64_t)gm * n + gn + 1] = __fadd_rn(acc[i][jj].s.y, acc[i][jj].c.y);
        }
    }
}

// C = alpha * sum_z partial[z] + beta * C, z ascending (deterministic split-K).
template <typename Tacc, typename Tout>
__global__ void k_splitk_reduce(int M, int N, int splits, Tacc alpha, const Tacc* partial, Tacc beta, Tout* C,
                                int64_t ldc, int upper) {
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < (int64_t)M * N;
         f += (int64_t)gridDim.x * blockDim.x) {
        const int gm = (int)(f / N), gn = (int)(f % N);
        if (upper && gm > gn) continue;
        Tacc s = Tacc(0);
        for (int z = 0; z < splits; ++z) s += partial[(int64_t)z * M * N + f];
        Tacc c = alpha * s;
        if (beta != Tacc(0)) c = fma(beta, (Tacc)C[(int64_t)gm * ldc + gn], c);
        C[(int64_t)gm * ldc + gn] = (Tout)c;
    }
}

// ---------------------------------------------------------------------------
// Diagonal block: Eqs. 3-4 on the b x b block at (k0, k0) of X (in place),
// then the inverse of the triangular factor (R_KK^{-1}, upper) into Rinv.
// One CTA of kDiagThreads threads.
//
// Factor, right-looking with the block in registers: thread t holds the
// TR x TC tile at rows (t / 16) TR.., columns (t % 16) TC.. of a 32 TR x
// 16 TC grid.  At step i every entry (r, c), r > i, receives its Eq. 4 term
// -r_ir r_ic, so each entry still collects its terms in the order k = 0, 1,
// ..., r-1 (the left-looking sum's order) before it is scaled by 1/r_rr.
// The owners of row i+1 publish it (double-buffered) right after their
// update, and the owner of entry (i+1, i+1) forms the next pivot (Eq. 3),
// so a step needs one barrier.  R_KK^{-1} is formed the same way (right-
// looking back substitution, rows from the last to the first).  A pivot
// <= 0 or non-finite sets *failed and info (1-based global row).
// ---------------------------------------------------------------------------
constexpr int kDiagThreads = 512;

template <typename T> struct DiagTile;
template <> struct DiagTile<float>  { static constexpr int TR = 4, TC = 8; };  // b <= 128
template <> struct DiagTile<double> { static constexpr int TR = 2, TC = 4; };  // b <= 64

template <typename T>
__global__ void __launch_bounds__(kDiagThreads)
k_blk_potrf(T* X, int64_t ldx, int n0, int k0, int b, T* Rinv, int* failed, int32_t* info, int pivot64) {
    constexpr int TR = DiagTile<T>::TR, TC = DiagTile<T>::TC;
    constexpr int BMAX = 16 * TC;  // = 32 * TR
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int LD = b + 1;
    T* Ro = reinterpret_cast<T*>(smem_raw);  // [b][LD]   R_KK (upper, zeros below)
    T* Pb = Ro + (size_t)b * LD;             // [2][BMAX]  pivot row (unscaled), double-buffered
    T* dv = Pb + 2 * BMAX;                   // [b]        1 / r_ii
    T* d0 = dv + b;                          // [b]        a_ii (FP64 pivots)
    __shared__ T s_piv[2][2];                // per parity: r_ii, 1 / r_ii
    __shared__ int s_bad[2];
    const int t = threadIdx.x;
    if (*failed) return;
    const int r0 = (t / 16) * TR, c0 = (t % 16) * TC;
    for (int f = t; f < 2 * BMAX; f += blockDim.x) Pb[f] = T(0);  // entries past b stay zero
    T a[TR][TC];
#pragma unroll
    for (int u = 0; u < TR; ++u)
#pragma unroll
        for (int v = 0; v < TC; ++v) {
            const int r = r0 + u, c = c0 + v;
            a[u][v] = (r <= c && c < b) ? X[(int64_t)(k0 + r) * ldx + k0 + c] : T(0);
            if (r == c && c < b) d0[r] = a[u][v];
        }
    // pivot of row `r` from its Schur value s (Eq. 3), into slot r & 1
    auto set_pivot = [&](int r, T s) {
        const bool bad = !(s > T(0)) || !isfinite(s);
        T rii, inv;
        pivot_root(s, rii, inv);
        s_bad[r & 1] = bad;
        s_piv[r & 1][0] = rii;
        s_piv[r & 1][1] = inv;
    };
    // FP64 form of Eq. 3 for row r: a_rr minus the exact squares of column r of R (warp 0)
    auto set_pivot64 = [&](int r) {
        double part = 0.0;
        for (int k = t; k < r; k += 32) part += (double)Ro[k * LD + r] * (double)Ro[k * LD + r];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) part += __shfl_xor_sync(0xffffffffu, part, d);
        if (t == 0) {
            const double td = (double)d0[r] - part;
            s_bad[r & 1] = !(td > 0.0) || !isfinite(td);
            s_piv[r & 1][0] = (T)sqrt(td);
            s_piv[r & 1][1] = (T)(1.0 / sqrt(td));
        }
    };
    const bool p64 = pivot64 && sizeof(T) == 4;
    __syncthreads();
    // row 0 published, its pivot formed
    if (r0 == 0) {
#pragma unroll
        for (int v = 0; v < TC; ++v)
            if (c0 + v < b) Pb[c0 + v] = a[0][v];
        if (c0 == 0 && !p64) set_pivot(0, a[0][0]);
    }
    __syncthreads();
    if (p64 && t < 32) set_pivot64(0);
    if (p64) __syncthreads();
    // ---------------- factor, Eqs. 3-4
    for (int i = 0; i < b; ++i) {
        const T* P = Pb + (i & 1) * BMAX;
        if (s_bad[i & 1]) {
            // every thread reads the same flag, so all of them leave here
            if (t == 0 && atomicCAS(failed, 0, 1) == 0 && info) *info = k0 + i + 1;
            return;
        }
        const T rii = s_piv[i & 1][0], inv = s_piv[i & 1][1];
        if (t < b) Ro[i * LD + t] = (t > i) ? P[t] * inv : (t == i ? rii : T(0));  // row i of R (Eq. 4)
        if (t == 0) dv[i] = inv;
        if (r0 + TR - 1 > i) {  // the tile has rows below the pivot row
            // Entries (r, c) with r <= i (rows already published) or c <= i
            // (below the diagonal of the rows still open) are never read
            // again, so the update runs over the whole tile unguarded; the
            // buffer's entries at and past b are zero, which keeps the tile's
            // columns past b at zero.
            T pr[TR], pc[TC];
#pragma unroll
            for (int u = 0; u < TR; ++u) pr[u] = P[r0 + u] * inv;
#pragma unroll
            for (int v = 0; v < TC; ++v) pc[v] = P[c0 + v] * inv;
#pragma unroll
            for (int u = 0; u < TR; ++u)
#pragma unroll
                for (int v = 0; v < TC; ++v) a[u][v] = fma(-pr[u], pc[v], a[u][v]);
            // publish row i+1 (final in the columns >= i+1) and form its pivot
            T* Pn = Pb + ((i + 1) & 1) * BMAX;
#pragma unroll
            for (int u = 0; u < TR; ++u) {
                if (r0 + u == i + 1) {
#pragma unroll
                    for (int v = 0; v < TC; ++v) Pn[c0 + v] = a[u][v];
                    if (!p64 && c0 <= i + 1 && i + 1 < c0 + TC) {
#pragma unroll
                        for (int v = 0; v < TC; ++v)
                            if (c0 + v == i + 1) set_pivot(i + 1, a[u][v]);
                    }
                }
            }
        }
        __syncthreads();
        if (p64 && i + 1 < b) {
            if (t < 32) set_pivot64(i + 1);
            __syncthreads();
        }
    }
    // R_KK back to X (upper part)
    for (int f = t; f < b * b; f += blockDim.x) {
        const int i = f / b, j = f % b;
        if (i <= j) X[(int64_t)(k0 + i) * ldx + k0 + j] = Ro[i * LD + j];
    }
    // ---------------- R_KK W = I, rows from the last to the first; the tile
    // holds B (W before each row's scaling by 1/r_kk)
#pragma unroll
    for (int u = 0; u < TR; ++u)
#pragma unroll
        for (int v = 0; v < TC; ++v) a[u][v] = (r0 + u == c0 + v) ? T(1) : T(0);
    __syncthreads();  // the factor's last reads of the buffer are done
#pragma unroll
    for (int u = 0; u < TR; ++u)
        if (r0 + u == b - 1) {
#pragma unroll
            for (int v = 0; v < TC; ++v) Pb[((b - 1) & 1) * BMAX + c0 + v] = a[u][v];
        }
    __syncthreads();
    for (int k = b - 1; k >= 0; --k) {
        const T* P = Pb + (k & 1) * BMAX;
        if (r0 < k) {  // the tile has rows above row k
            const T dk = dv[k];
            // rows >= k keep their values (row k is final); the published row
            // is exactly zero left of its diagonal and past b
            T rk[TR], wk[TC];
#pragma unroll
            for (int u = 0; u < TR; ++u) rk[u] = (r0 + u < k) ? Ro[(r0 + u) * LD + k] : T(0);
#pragma unroll
            for (int v = 0; v < TC; ++v) wk[v] = P[c0 + v] * dk;
#pragma unroll
            for (int u = 0; u < TR; ++u)
#pragma unroll
                for (int v = 0; v < TC; ++v) a[u][v] = fma(-rk[u], wk[v], a[u][v]);
            T* Pn = Pb + ((k - 1) & 1) * BMAX;
#pragma unroll
            for (int u = 0; u < TR; ++u)
                if (r0 + u == k - 1) {
#pragma unroll
                    for (int v = 0; v < TC; ++v) Pn[c0 + v] = a[u][v];
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < TR; ++u)
#pragma unroll
        for (int v = 0; v < TC; ++v) {
            const int r = r0 + u, c = c0 + v;
            if (r < b && c < b) Rinv[(int64_t)r * b + c] = (r <= c) ? a[u][v] * dv[r] : T(0);
        }
}

// ---------------------------------------------------------------------------
// Diagonal block, blocked form (no FP64-pivot mode): the b x b block is split
// into 32 x 32 sub-blocks (padded with the identity up to a multiple of 32).
// For each sub-block row p:
//   leaf     one warp factors the diagonal sub-block A_pp (Eqs. 3-4,
//            right-looking, lane j holds column j in registers, rows of R
//            passed by shuffles) and forms W_pp = R_pp^{-1} by back
//            substitution;
//   panel    one warp per 32 columns to the right solves R_pp^T R_pq = A_pq
//            (Eq. 4 for the sub-block row: each entry receives its terms in
//            ascending k, then the scaling by 1/r_ii);
//   trailing the CTA applies A_qr -= R_pq^T R_pr (terms in ascending k);
// then the off-diagonal blocks of W = R_KK^{-1} follow bottom-up,
// W_pq = -W_pp sum_{p<k<=q} R_pk W_kq.  About 16 CTA barriers in all, against
// 256 for the row-by-row kernel.
// ---------------------------------------------------------------------------
constexpr int kSB = 32;

template <typename T>
__global__ void __launch_bounds__(kDiagThreads)
k_blk_potrf_blk(T* X, int64_t ldx, int k0, int b, T* Rinv, int* failed, int32_t* info, int pivot64) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int NSB = (b + kSB - 1) / kSB;
    const int B = NSB * kSB;
    const int LD = B + 1;
    // pivot64: ds[j] = a_jj - sum_k r_kj^2 over the block's finished rows k,
    // in FP64 from exact products of the FP32 values (Eq. 3's in-block terms)
    double* ds = reinterpret_cast<double*>(smem_raw);  // [B]
    T* S = reinterpret_cast<T*>(ds + B);    // [B][LD] A, then R (upper)
    T* W = S + (size_t)B * LD;              // [B][LD] R^{-1} (upper); its lower blocks hold scratch
    T* dv = W + (size_t)B * LD;             // [B] 1 / r_ii
    __shared__ int s_bad;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    if (*failed) return;
    for (int f = t; f < B * B; f += blockDim.x) {
        const int i = f / B, j = f % B;
        T v;
        if (i < b && j < b) v = (i <= j) ? X[(int64_t)(k0 + i) * ldx + k0 + j] : T(0);
        else v = (i == j) ? T(1) : T(0);
        S[i * LD + j] = v;
        W[i * LD + j] = T(0);
        if (i == j) ds[i] = (double)v;
    }
    if (t == 0) s_bad = 0;
    __syncthreads();
    for (int p = 0; p < NSB; ++p) {
        const int o = p * kSB;
        // ---------------- leaf (warp 0)
        if (warp == 0) {
            T a[kSB];
#pragma unroll
            for (int k = 0; k < kSB; ++k) a[k] = S[(o + k) * LD + o + lane];
            int bad = 0;
            // pivot64: lane j's Eq. 3 argument in FP64, a_jj less r_kj^2 over
            // the rows k finished so far (one term per row, k ascending)
            double dl = pivot64 ? ds[o + lane] : 0.0;
#pragma unroll
            for (int i = 0; i < kSB; ++i) {
                const T tt = __shfl_sync(0xffffffffu, a[i], i);  // Eq. 3 argument (row i, column i)
                T rii, inv;
                if (pivot64) {
                    const double td = __shfl_sync(0xffffffffu, dl, i);
                    if (!bad && !(td > 0.0 && isfinite(td))) bad = o + i + 1;
                    pivot_root64(td, rii, inv);
                } else {
                    if (!bad && !(tt > T(0) && isfinite(tt))) bad = o + i + 1;
                    pivot_root(tt, rii, inv);
                }
                if (lane == i) a[i] = rii;
                else if (lane > i) a[i] = a[i] * inv;  // r_ij, Eq. 4
                if (pivot64 && lane > i) dl -= (double)a[i] * (double)a[i];
                if (lane == 0) dv[o + i] = inv;
#pragma unroll
                for (int k = 0; k < kSB; ++k) {  // fixed trip count: every index stays a constant
                    if (k > i) {
                        const T rik = __shfl_sync(0xffffffffu, a[i], k);
                        if (lane >= k) a[k] = fma(-rik, a[i], a[k]);
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < kSB; ++k)
                if (k <= lane) S[(o + k) * LD + o + lane] = a[k];
            __syncwarp();
            // W_pp = R_pp^{-1}, column `lane`, rows from the last to the first
            T w[kSB];
#pragma unroll
            for (int k = kSB - 1; k >= 0; --k) {
                T acc = (k == lane) ? T(1) : T(0);
#pragma unroll
                for (int m = 0; m < kSB; ++m)
                    if (m > k) acc = fma(-S[(o + k) * LD + o + m], w[m], acc);
                w[k] = acc * dv[o + k];
            }
#pragma unroll
            for (int k = 0; k < kSB; ++k) W[(o + k) * LD + o + lane] = w[k];
            if (lane == 0 && bad) s_bad = bad;
        }
        __syncthreads();
        if (s_bad) {
            if (t == 0 && s_bad <= b && atomicCAS(failed, 0, 1) == 0 && info) *info = k0 + s_bad;
            return;  // every thread reads the same flag
        }
        if (p + 1 == NSB) break;
        // ---------------- panel: warp w takes columns o + 32 (w + 1) + lane
        if (warp < NSB - 1 - p) {
            const int c = o + kSB * (warp + 1) + lane;
            T a[kSB];
#pragma unroll
            for (int k = 0; k < kSB; ++k) a[k] = S[(o + k) * LD + c];
#pragma unroll
            for (int i = 0; i < kSB; ++i) {
                T s = a[i];
#pragma unroll
                for (int k = 0; k < kSB; ++k)
                    if (k < i) s = fma(-S[(o + k) * LD + o + i], a[k], s);
                a[i] = s * dv[o + i];
            }
#pragma unroll
            for (int k = 0; k < kSB; ++k) S[(o + k) * LD + c] = a[k];
        }
        __syncthreads();
        if (pivot64) {
            // the sub-block's rows of R, column by column, off the later pivots' arguments
            for (int j = o + kSB + t; j < B; j += blockDim.x) {
                double d = ds[j];
                for (int k = o; k < o + kSB; ++k) d -= (double)S[k * LD + j] * (double)S[k * LD + j];
                ds[j] = d;
            }
        }
        // ---------------- trailing update of rows/columns past o + 32: 4 x 4 patches
        {
            const int r0 = o + kSB, n = B - r0;  // trailing order (a multiple of 32)
            const int np = n / 4;                 // patches per side
            for (int f = t; f < np * np; f += blockDim.x) {
                const int pr = f / np, pc = f % np;
                if (pr > pc) continue;  // below the diagonal: not needed
                const int rr = r0 + 4 * pr, cc = r0 + 4 * pc;
                T acc[4][4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[u][v] = S[(rr + u) * LD + cc + v];
#pragma unroll 4
                for (int k = 0; k < kSB; ++k) {
                    T x[4], y[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) x[u] = S[(o + k) * LD + rr + u];
#pragma unroll
                    for (int v = 0; v < 4; ++v) y[v] = S[(o + k) * LD + cc + v];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int v = 0; v < 4; ++v) acc[u][v] = fma(-x[u], y[v], acc[u][v]);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) S[(rr + u) * LD + cc + v] = acc[u][v];
            }
        }
        __syncthreads();
    }
    // R_KK back to X (upper part)
    for (int f = t; f < b * b; f += blockDim.x) {
        const int i = f / b, j = f % b;
        if (i <= j) X[(int64_t)(k0 + i) * ldx + k0 + j] = S[i * LD + j];
    }
    // ---------------- off-diagonal blocks of W, bottom-up
    for (int p = NSB - 2; p >= 0; --p) {
        const int o = p * kSB, r0 = o + kSB, n = B - r0;
        // T_q = R_p,(p,q] W_(p,q],q for every column c >= r0, into W's lower block
        // rows (its rows r0 + i, i < 32, columns o.. hold nothing else)
        for (int f = t; f < kSB * n; f += blockDim.x) {
            const int i = f / n, c = r0 + f % n;
            T acc = T(0);
            for (int m = r0; m <= c; ++m) acc = fma(S[(o + i) * LD + m], W[m * LD + c], acc);
            W[(c) * LD + o + i] = acc;  // transposed into the strictly lower part (c > o + i)
        }
        __syncthreads();
        // W_pq = -W_pp T_q
        for (int f = t; f < kSB * n; f += blockDim.x) {
            const int i = f / n, c = r0 + f % n;
            T acc = T(0);
#pragma unroll 8
            for (int k = 0; k < kSB; ++k) acc = fma(W[(o + i) * LD + o + k], W[c * LD + o + k], acc);
            W[(o + i) * LD + c] = -acc;
        }
        __syncthreads();
    }
    for (int f = t; f < b * b; f += blockDim.x) {
        const int i = f / b, j = f % b;
        Rinv[(int64_t)i * b + j] = (i <= j) ? W[i * LD + j] : T(0);
    }
}

// ---------------------------------------------------------------------------
// Diagonal block of X, Sec. IV.A in block form.  Row block I of R X = S
// (S lower triangular with diagonal 1/r_ii; its diagonal block is R_II^{-T})
// gives, with W = R_II^{-1} and Z = R_I,>I X_>I,I (= R_I,>I X_I,>I^T):
//   X_II = W (W^T - Z),
// the block counterpart of x_ii = (1/r_ii)(1/r_ii - sum_{k>i} r_ik x_ik) and
// x_ij = -(1/r_ii) sum_{k>i} r_ik x~_kj.  One CTA per 32 x 32 tile on or above
// the block's diagonal; each result is written to both triangles (on a
// diagonal tile only the entries with i <= j are written, and mirrored).
// ---------------------------------------------------------------------------
constexpr int kXdT = 32;

template <typename T>
__global__ void __launch_bounds__(256)
k_blk_xdiag(T* X, int64_t ldx, int i0, int b, const T* W, const T* Z, const int* failed) {
    __shared__ T Ws[kXdT][kXdT + 1];  // W[i][k]
    __shared__ T Ys[kXdT][kXdT + 1];  // W[j][k] - Z[k][j]
    const int ti = blockIdx.y, tj = blockIdx.x;
    if (ti > tj || *failed) return;
    const int t = threadIdx.x;
    const int ri = t / 8, cj = (t % 8) * 4;  // one row, four columns of the tile
    const int ib = ti * kXdT, jb = tj * kXdT;
    T acc[4] = {T(0), T(0), T(0), T(0)};
    for (int kb = ib; kb < b; kb += kXdT) {  // W[i][k] = 0 for k < i
        for (int f = t; f < kXdT * kXdT; f += 256) {
            const int x = f / kXdT, y = f % kXdT;
            const int i = ib + x, k = kb + y;
            Ws[x][y] = (i < b && k < b && k >= i) ? W[(int64_t)i * b + k] : T(0);
            const int kk = kb + x, j = jb + y;
            T yv = T(0);
            if (kk < b && j < b) {
                yv = (kk >= j) ? W[(int64_t)j * b + kk] : T(0);
                if (Z) yv -= Z[(int64_t)kk * b + j];
            }
            Ys[x][y] = yv;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < kXdT; ++k) {
            const T w = Ws[ri][k];
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[c] = fma(w, Ys[k][cj + c], acc[c]);
        }
        __syncthreads();
    }
    const int i = ib + ri;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int j = jb + cj + c;
        if (i >= b || j >= b || (ti == tj && i > j)) continue;
        X[(int64_t)(i0 + i) * ldx + i0 + j] = acc[c];
        if (i != j) X[(int64_t)(i0 + j) * ldx + i0 + i] = acc[c];
    }
}

// Copy a b x m panel P into X at (r0, c0) and its transpose at (c0, r0).
template <typename T>
__global__ void k_put_panel(T* X, int64_t ldx, int r0, int c0, int b, int m, const T* P, int mirror, const int* failed) {
    if (*failed) return;
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < (int64_t)b * m;
         f += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(f / m), j = (int)(f % m);
        const T v = P[f];
        X[(int64_t)(r0 + i) * ldx + c0 + j] = v;
        if (mirror) X[(int64_t)(c0 + j) * ldx + r0 + i] = v;
    }
}

// Copy the transpose of an m x b panel Pt into X at (r0, c0) (X[r0+i][c0+j] = Pt[j][i]).
__global__ void k_put_panel_t(float* X, int64_t ldx, int r0, int c0, int b, int m, const float* Pt, const int* failed) {
    if (*failed) return;
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < (int64_t)b * m;
         f += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(f / m), j = (int)(f % m);
        X[(int64_t)(r0 + i) * ldx + c0 + j] = Pt[(int64_t)j * b + i];
    }
}

// A tensor-core GEMM gave up waiting: report it, and make the result NaN.
__global__ void k_report_umma(const int* umma_err, int* failed, int* err_word) {
    if (*umma_err) {
        atomicCAS(err_word, 0, CHOL_ERR_TIMEOUT);
        *failed = 1;
    }
}

// X (n x n) <- upper triangle of A (layout dense, ld n); lower part cleared.
template <typename T>
__global__ void k_load_upper(T* X, const T* A, int n) {
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < (int64_t)n * n;
         f += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(f / n), j = (int)(f % n);
        X[f] = (i <= j) ? A[f] : T(0);
    }
}

// Full symmetric copy of A from its upper triangle (for the refinement residual).
template <typename T>
__global__ void k_sym_full(T* F, const T* A, int n) {
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < (int64_t)n * n;
         f += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(f / n), j = (int)(f % n);
        F[f] = (i <= j) ? A[f] : A[(int64_t)j * n + i];
    }
}

template <typename T>
__global__ void k_identity(T* E, int n) {
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < (int64_t)n * n;
         f += (int64_t)gridDim.x * blockDim.x)
        E[f] = ((f / n) == (f % n)) ? T(1) : T(0);
}

// Fill X with NaN when the factorisation failed.
template <typename T>
__global__ void k_nan_if_failed(T* X, int64_t count, const int* failed) {
    if (!*failed) return;
    const T q = T(__int_as_float(0x7fffffff));
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < count; f += (int64_t)gridDim.x * blockDim.x)
        X[f] = q;
}

// X += C elementwise.
__global__ void k_axpy(float* X, const float* C, int64_t count) {
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < count; f += (int64_t)gridDim.x * blockDim.x)
        X[f] += C[f];
}

// R <- upper triangle of X, lower part zero (the factor, before the inverse overwrites it).
template <typename T>
__global__ void k_copy_upper(T* R, const T* X, int n, const int* failed) {
    const T q = T(__int_as_float(0x7fffffff));
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < (int64_t)n * n;
         f += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(f / n), j = (int)(f % n);
        R[f] = *failed ? q : ((i <= j) ? X[f] : T(0));
    }
}

// Complex Hermitian A = B + iC (B symmetric, C = Im A antisymmetric) as the
// real symmetric matrix M = [[B, -C], [C, B]] of order 2n (M [x; y] is A z
// for z = x + iy): M is positive definite exactly when A is, and
// M^{-1} = [[P, -Q], [Q, P]] for A^{-1} = P + iQ.  Only A's upper triangle is
// read (its diagonal taken as real); M is written in full.  32 x 32 tiles,
// those below the diagonal read transposed through shared memory.
constexpr int kEmT = 32;
template <typename R>
__global__ void __launch_bounds__(kEmT * 8) k_embed_hermitian(const cpx<R>* __restrict__ A, R* __restrict__ M,
                                                               int n) {
    __shared__ cpx<R> tile[kEmT][kEmT + 1];
    const int ti = blockIdx.y, tj = blockIdx.x;
    const bool up = ti <= tj;  // the source tile: (ti, tj) on or above the diagonal, else (tj, ti)
    const int si = up ? ti : tj, sj = up ? tj : ti;
    const int c = threadIdx.x;
    for (int r = threadIdx.y; r < kEmT; r += blockDim.y) {
        const int i = si * kEmT + r, j = sj * kEmT + c;
        tile[r][c] = (i < n && j < n) ? A[(int64_t)i * n + j] : cpx<R>{R(0), R(0)};
    }
    __syncthreads();
    const int64_t L = 2 * (int64_t)n;
    for (int r = threadIdx.y; r < kEmT; r += blockDim.y) {
        const int i = ti * kEmT + r, j = tj * kEmT + c;
        if (i >= n || j >= n) continue;
        // a_ij from the upper triangle: a_ij itself, or conj(a_ji) below the diagonal
        const cpx<R> a = (i <= j) ? tile[r][c] : conj_v(tile[c][r]);
        const R im = (i == j) ? R(0) : a.im;
        M[i * L + j] = a.re;
        M[(n + i) * L + n + j] = a.re;
        M[i * L + n + j] = -im;
        M[(n + i) * L + j] = im;
    }
}

// X = P + iQ from the inverse of the embedding (full, dense): P its top-left
// block, Q the mean of its bottom-left block and the negated top-right one
// (equal but for rounding), each entry below the diagonal the conjugate of
// its mirror, so that X is exactly Hermitian with a real diagonal.
template <typename R>
__global__ void k_extract_hermitian(const R* __restrict__ XM, cpx<R>* __restrict__ X, int n) {
    const int64_t L = 2 * (int64_t)n;
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < (int64_t)n * n;
         f += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = f / n, c = f - r * n;
        const int64_t i = r < c ? r : c, j = r < c ? c : r;  // the upper-triangle entry (i <= j)
        const R q = (i == j) ? R(0) : R(0.5) * (XM[(n + i) * L + j] - XM[i * L + n + j]);
        X[f] = {XM[i * L + j], r <= c ? q : -q};
    }
}

// Convert the FP64 residual to the working precision.
__global__ void k_narrow(float* dst, const double* src, int64_t count) {
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < count; f += (int64_t)gridDim.x * blockDim.x)
        dst[f] = (float)src[f];
}

// ---------------------------------------------------------------------------
// Host driver
// ---------------------------------------------------------------------------
namespace {

// Panel width b: 128 for FP32, 64 for FP64 (the diagonal-block kernels hold
// two b x b blocks in shared memory).
constexpr int kblk(int dtype) { return dtype == CHOL_F64 ? 64 : 128; }

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

struct BlkWs {
    char* base;
    size_t off = 0;
    template <typename U>
    U* take(size_t count) {
        U* p = reinterpret_cast<U*>(base + off);
        off += align256(count * sizeof(U));
        return p;
    }
};

template <typename Tin, typename Tacc, typename Tout, bool TA, bool TB>
cudaError_t gemm(int M, int N, int K, Tacc alpha, const Tin* A, int64_t lda, const Tin* B, int64_t ldb, Tacc beta,
                 Tout* C, int64_t ldc, int upper, Tacc* partial, size_t partial_elems, cudaStream_t s) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    const int sms = device_info().sms;
    dim3 grid((N + GB_N - 1) / GB_N, (M + GB_M - 1) / GB_M, 1);
    int splits = 1;
    if (partial && K > 0) {
        const int tiles = grid.x * grid.y;
        // split K until the grid covers the SMs twice, keeping >= 32 of K per slice
        while (splits < 32 && tiles * splits * 2 <= 2 * sms && K / (splits * 2) >= 32 &&
               (size_t)M * N * splits * 2 <= partial_elems)
            splits *= 2;
    }
    if (splits == 1) {
        k_gemm<Tin, Tacc, Tout, TA, TB><<<grid, GB_THREADS, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc,
                                                                   upper, K > 0 ? K : 1, nullptr);
        return cudaGetLastError();
    }
    int kchunk = (K + splits - 1) / splits;
    kchunk = (kchunk + GB_K - 1) / GB_K * GB_K;
    grid.z = splits;
    k_gemm<Tin, Tacc, Tacc, TA, TB><<<grid, GB_THREADS, 0, s>>>(M, N, K, Tacc(1), A, lda, B, ldb, Tacc(0),
                                                               partial, N, upper, kchunk, partial);
    const int64_t total = (int64_t)M * N;
    const int rgrid = (int)std::min<int64_t>((total + 255) / 256, (int64_t)sms * 8);
    k_splitk_reduce<Tacc, Tout><<<rgrid, 256, 0, s>>>(M, N, splits, alpha, partial, beta, C, ldc, upper);
    return cudaGetLastError();
}

}  // namespace

// ---------------------------------------------------------------------------
// Tensor-core GEMM host side: TMA tensor maps and launches.
// ---------------------------------------------------------------------------
namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// Row-major FP32 matrix (rows x cols, leading dimension ld elements) as a 2-D
// tensor map with 32 x 128 boxes and the 128-byte swizzle; entries outside
// the matrix read as zero.
bool make_map(CUtensorMap* m, const float* base, int64_t rows, int64_t cols, int64_t ld) {
    EncodeTiledFn enc = encode_fn();
    if (!enc || (reinterpret_cast<uintptr_t>(base) & 15) || (ld * 4) % 16) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * 4)};
    cuuint32_t box[2] = {(cuuint32_t)umma::BK, (cuuint32_t)umma::BM};
    cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int STAGES, int SPLIT3, int CPRE>
cudaError_t umma_setup() {
    static std::once_flag once;
    static cudaError_t e = cudaSuccess;
    std::call_once(once, [] {
        e = cudaFuncSetAttribute(umma::k_umma_gemm<STAGES, SPLIT3, CPRE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)umma::smem_bytes<STAGES, SPLIT3, CPRE>());
    });
    return e;
}

// C = alpha A B^T + beta C on the tensor cores (A: M x K at map coordinates
// (ax, ay); B: N x K at (bx, by)); split-K through `partial` when the tile
// grid alone would leave most of the GPU idle.
cudaError_t umma_gemm(int M, int N, int K, float alpha, const CUtensorMap& ma, int ax, int ay, const CUtensorMap& mb,
                      int bx, int by, float beta, float* C, int64_t ldc, int upper, float* partial, size_t partial_elems,
                      int split3, int* err, cudaStream_t s) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    const int sms = device_info().sms;
    dim3 grid((N + umma::BN - 1) / umma::BN, (M + umma::BM - 1) / umma::BM, 1);
    int splits = 1;
    const int tiles = grid.x * grid.y;
    while (partial && splits < 32 && tiles * splits * 2 <= sms && K / (splits * 2) >= 4 * umma::BK &&
           (size_t)M * N * splits * 2 <= partial_elems)
        splits *= 2;
    umma::GemmArgs g;
    g.M = M; g.N = N; g.K = K;
    g.ax = ax; g.ay = ay; g.bx = bx; g.by = by;
    g.alpha = alpha; g.beta = beta; g.C = C; g.ldc = ldc; g.upper = upper;
    int kchunk = (K + splits - 1) / splits;
    kchunk = (kchunk + umma::BK - 1) / umma::BK * umma::BK;
    g.kchunk = kchunk;
    g.partial = splits > 1 ? partial : nullptr;
    g.split3 = split3;
    g.err = err;
    grid.z = splits;
    // C prefetched by bulk copies when it is read (beta != 0, no split-K) and
    // its rows are 16-byte aligned; two stages then leave room for the C tile
    const bool cpre = beta != 0.f && splits == 1 && ldc % 4 == 0 && N % 4 == 0 &&
                      reinterpret_cast<uintptr_t>(C) % 16 == 0;
    cudaError_t e;
    if (split3 && cpre) {
        if ((e = umma_setup<2, 1, 1>()) != cudaSuccess) return e;
        umma::k_umma_gemm<2, 1, 1><<<grid, umma::THREADS, umma::smem_bytes<2, 1, 1>(), s>>>(ma, mb, g);
    } else if (split3) {
        if ((e = umma_setup<3, 1, 0>()) != cudaSuccess) return e;
        umma::k_umma_gemm<3, 1, 0><<<grid, umma::THREADS, umma::smem_bytes<3, 1, 0>(), s>>>(ma, mb, g);
    } else if (cpre) {
        if ((e = umma_setup<4, 0, 1>()) != cudaSuccess) return e;
        umma::k_umma_gemm<4, 0, 1><<<grid, umma::THREADS, umma::smem_bytes<4, 0, 1>(), s>>>(ma, mb, g);
    } else {
        if ((e = umma_setup<4, 0, 0>()) != cudaSuccess) return e;
        umma::k_umma_gemm<4, 0, 0><<<grid, umma::THREADS, umma::smem_bytes<4, 0, 0>(), s>>>(ma, mb, g);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (splits > 1) {
        const int64_t total = (int64_t)M * N;
        const int rgrid = (int)std::min<int64_t>((total + 255) / 256, (int64_t)sms * 8);
        k_splitk_reduce<float, float><<<rgrid, 256, 0, s>>>(M, N, splits, alpha, partial, beta, C, ldc, upper);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace

namespace {
// A side stream (per device) for the factor's lookahead, with the two events
// that fork it from and join it to the caller's stream.  Enqueueing holds
// the mutex, so concurrent calls on one device take turns at it.
struct SideStream {
    cudaStream_t s = nullptr;
    cudaEvent_t ready = nullptr, done = nullptr;
    std::mutex mu;
};
SideStream* side_stream() {
    static std::mutex init_mu;
    static SideStream* per_dev[64] = {};
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(init_mu);
    if (!per_dev[d]) {
        SideStream* ss = new SideStream();
        if (cudaStreamCreateWithFlags(&ss->s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ss->ready, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&ss->done, cudaEventDisableTiming) != cudaSuccess) {
            delete ss;
            return nullptr;
        }
        per_dev[d] = ss;
    }
    return per_dev[d];
}
}  // namespace

// ---------------------------------------------------------------------------
// Kernel timing of the blocked path (chol_blocked_timing*): while enabled on
// a host thread, the calls it makes record an event pair around each product
// of the kinds below on the stream that runs it, with the product's
// algorithmic flops (2 M N K; the upper half only where only it is formed).
// ---------------------------------------------------------------------------
struct BlkTiming {
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[kBlkTimingKinds];
    double flops[kBlkTimingKinds] = {};
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    cudaEvent_t take() {
        if (used == pool.size()) {
            cudaEvent_t e = nullptr;
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
            pool.push_back(e);
        }
        return pool[used++];
    }
};
thread_local BlkTiming* t_blk = nullptr;

// f() bracketed by an event pair of `kind` when timing is on.
template <class F>
cudaError_t timed(int kind, double flops, cudaStream_t s, F&& f) {
    BlkTiming* t = t_blk;
    cudaEvent_t e0 = t ? t->take() : nullptr, e1 = t ? t->take() : nullptr;
    if (t && e0 && e1 && cudaEventRecord(e0, s) != cudaSuccess) return cudaGetLastError();
    cudaError_t e = f();
    if (e != cudaSuccess) return e;
    if (t && e0 && e1) {
        if ((e = cudaEventRecord(e1, s)) != cudaSuccess) return e;
        t->ev[kind].push_back({e0, e1});
        t->flops[kind] += flops;
    }
    return cudaSuccess;
}

// Algorithmic flops of an M x N product with inner dimension K whose region
// starts on the diagonal and keeps only its upper part (upper != 0).
double gemm_flops(int M, int N, int K, int upper) {
    if (!upper) return 2.0 * M * N * K;
    const double rows = std::min(M, N);
    return 2.0 * K * (rows * N - rows * (rows - 1) / 2);
}

void blocked_timing_enable(int on) {
    if (on) {
        if (!t_blk) t_blk = new BlkTiming();
        for (int k = 0; k < kBlkTimingKinds; ++k) {
            t_blk->ev[k].clear();
            t_blk->flops[k] = 0;
        }
        t_blk->used = 0;
    } else if (t_blk) {
        for (cudaEvent_t e : t_blk->pool) cudaEventDestroy(e);
        delete t_blk;
        t_blk = nullptr;
    }
}

cudaError_t blocked_timing_read(int kind, float* ms, double* flops, int* launches) {
    *ms = 0.f;
    *flops = 0.0;
    *launches = 0;
    if (!t_blk || kind < 0 || kind >= kBlkTimingKinds) return cudaErrorInvalidValue;
    for (auto& pr : t_blk->ev[kind]) {
        cudaError_t e = cudaEventSynchronize(pr.second);
        if (e != cudaSuccess) return e;
        float m = 0.f;
        if ((e = cudaEventElapsedTime(&m, pr.first, pr.second)) != cudaSuccess) return e;
        *ms += m;
    }
    *flops = t_blk->flops[kind];
    *launches = (int)t_blk->ev[kind].size();
    return cudaSuccess;
}

size_t blocked_workspace_bytes(int dtype, int n, int refine) {
    if (n <= 0) return 0;
    if (dtype == CHOL_C64 || dtype == CHOL_C128) {
        // the real embedding of order 2n and its inverse, then the real path's own
        const int real = dtype == CHOL_C64 ? CHOL_F32 : CHOL_F64;
        const size_t es = dtype == CHOL_C64 ? 4 : 8;
        return 2 * align256((size_t)4 * n * n * es) + blocked_workspace_bytes(real, 2 * n, refine);
    }
    const size_t es = (dtype == CHOL_F64) ? 8 : 4;
    const int kBlk = kblk(dtype);
    const int nb = (n + kBlk - 1) / kBlk;
    size_t bytes = 256;                                       // failed flag
    bytes += align256((size_t)nb * kBlk * kBlk * es);         // Rinv blocks
    bytes += 3 * align256((size_t)kBlk * n * es);             // panels (one double-buffered)
    bytes += align256((size_t)kBlk * kBlk * es);              // Z
    bytes += align256((size_t)32 * kBlk * n * (dtype == CHOL_F64 ? 8 : 4));  // split-K partials
    bytes += align256((size_t)8 * kBlk * n * (dtype == CHOL_F64 ? 8 : 4));   // side stream's partials
    bytes += 256;                                                             // tensor-core error flag
    if (refine) {
        bytes += align256((size_t)n * n * 4);   // full A (FP32)
        bytes += align256((size_t)n * n * 8);   // residual (FP64)
        bytes += align256((size_t)n * n * 4);   // residual (FP32) / correction
        bytes += align256((size_t)32 * std::max<size_t>((size_t)n * n, 1) * 0);  // (no extra partials)
    }
    return bytes;
}

template <typename T>
static chol_status_t blocked_one(const T* A, T* R, T* X, int n, int32_t* info, int pivot64, int refine_steps,
                                 int resid64, int want_inv, int tc, int* err_word, char* ws, cudaStream_t s) {
    using Tacc = T;
    const int b = kblk(sizeof(T) == 8 ? CHOL_F64 : CHOL_F32);
    const int nb = (n + b - 1) / b;
    BlkWs w{ws};
    int* failed = w.take<int>(64);
    T* Rinv = w.take<T>((size_t)nb * b * b);
    T* P = w.take<T>((size_t)b * n);
    T* P2 = w.take<T>((size_t)b * n);
    T* P3 = w.take<T>((size_t)b * n);
    T* Z = w.take<T>((size_t)b * b);
    const size_t part_elems = (size_t)32 * b * n;
    Tacc* part = w.take<Tacc>(part_elems);
    const size_t part2_elems = (size_t)8 * b * n;
    Tacc* part2 = w.take<Tacc>(part2_elems);
    int* umma_err = w.take<int>(64);
    const int sms = device_info().sms;
    // tensor cores for the two large products (trailing update, inverse
    // assembly): FP32 only, and the tensor maps need 16-byte rows
    CUtensorMap mapX, mapPt[2];
    bool use_tc = tc != 0 && sizeof(T) == 4 && n % 4 == 0 && b % 4 == 0;
    if (use_tc)
        use_tc = make_map(&mapX, reinterpret_cast<const float*>(X), n, n, n) &&
                 make_map(&mapPt[0], reinterpret_cast<const float*>(P2), n, b, b) &&
                 make_map(&mapPt[1], reinterpret_cast<const float*>(P3), n, b, b);
    const int split3 = tc == 2 ? 1 : 0;
    const int g1 = sms * 4;
    static std::once_flag once;
    static cudaError_t setup = cudaSuccess;
    const size_t potrf_smem = ((size_t)b * (b + 1) + 2 * (size_t)16 * DiagTile<T>::TC + 2 * (size_t)b) * sizeof(T);
    const size_t potrf_blk_smem = (2 * (size_t)b * (b + 1) + (size_t)b) * sizeof(T) + (size_t)b * sizeof(double);
    std::call_once(once, [&] {
        setup = cudaFuncSetAttribute(k_blk_potrf<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)potrf_smem);
        if constexpr (sizeof(T) == 4)
            if (setup == cudaSuccess)
                setup = cudaFuncSetAttribute(k_blk_potrf_blk<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)potrf_blk_smem);
    });
    if (setup != cudaSuccess) return CHOL_ERR_CUDA;
    if (cudaMemsetAsync(failed, 0, sizeof(int), s) != cudaSuccess) return CHOL_ERR_CUDA;
    if (cudaMemsetAsync(umma_err, 0, sizeof(int), s) != cudaSuccess) return CHOL_ERR_CUDA;
    if (info && cudaMemsetAsync(info, 0, sizeof(int32_t), s) != cudaSuccess) return CHOL_ERR_CUDA;
    k_load_upper<T><<<g1, 256, 0, s>>>(X, A, n);
    // ---------------- factor, with one block of lookahead: once the trailing
    // update has reached block row K+1, that block's diagonal factor and
    // panel (the critical path) run on a side stream while the main stream
    // updates the remaining rows.  Panels alternate between two buffers.
    T* pbuf[2] = {use_tc ? P2 : P, P3};
    // R_KK and R_K,>K of block kb into X; the panel, in the layout the
    // trailing update reads, into pbuf[kb & 1]
    auto panel = [&](int kb, cudaStream_t st, Tacc* pw, size_t pw_elems) -> cudaError_t {
        const int k0 = kb * b;
        const int bk = std::min(b, n - k0);
        const int m = n - k0 - bk;
        T* RinvK = Rinv + (size_t)kb * b * b;
        // FP32: the blocked diagonal factor; FP64 (whose 32-wide register
        // columns do not fit) and FP64 pivots: the row-by-row one
        bool blk = false;
        if constexpr (sizeof(T) == 4) blk = true;  // FP32: the sub-block factor, FP64 pivots in it on request
        if (blk) {
            if constexpr (sizeof(T) == 4)
                k_blk_potrf_blk<T><<<1, kDiagThreads, potrf_blk_smem, st>>>(X, n, k0, bk, RinvK, failed, info,
                                                                            pivot64);
        } else {
            k_blk_potrf<T><<<1, kDiagThreads, potrf_smem, st>>>(X, n, n, k0, bk, RinvK, failed, info, pivot64);
        }
        if (m <= 0) return cudaGetLastError();
        T* pb = pbuf[kb & 1];
        if (use_tc) {
            // Pt = A_K,>K^T R_KK^{-1} = (R_K,>K)^T (m x bk, K-major for the tensor cores)
            cudaError_t e = gemm<T, Tacc, T, true, false>(m, bk, bk, Tacc(1), X + (int64_t)k0 * n + k0 + bk, n, RinvK,
                                                          bk, Tacc(0), pb, bk, 0, pw, pw_elems, st);
            if (e != cudaSuccess) return e;
            if constexpr (sizeof(T) == 4) k_put_panel_t<<<g1, 256, 0, st>>>(X, n, k0, k0 + bk, bk, m, pb, failed);
        } else {
            // R_K,>K = R_KK^{-T} A_K,>K  (bk x m, ld m), then back into X
            cudaError_t e = gemm<T, Tacc, T, true, false>(bk, m, bk, Tacc(1), RinvK, bk, X + (int64_t)k0 * n + k0 + bk,
                                                          n, Tacc(0), pb, m, 0, pw, pw_elems, st);
            if (e != cudaSuccess) return e;
            k_put_panel<T><<<g1, 256, 0, st>>>(X, n, k0, k0 + bk, bk, m, pb, 0, failed);
        }
        return cudaGetLastError();
    };
    // A_>K,>K -= R_K,>K^T R_K,>K on rows [r0, r1) of the trailing matrix
    // (columns >= each row: upper part)
    auto update = [&](int kb, int r0, int r1) -> cudaError_t {
        const int k0 = kb * b;
        const int bk = std::min(b, n - k0);
        const int m = n - k0 - bk;
        if (r1 <= r0) return cudaSuccess;
        T* Ct = X + (int64_t)(k0 + bk + r0) * n + k0 + bk + r0;
        T* pb = pbuf[kb & 1];
        if constexpr (sizeof(T) == 4) {
            if (use_tc)
                return timed(kBlkTrailingUpdate, gemm_flops(r1 - r0, m - r0, bk, 1), s, [&] {
                    return umma_gemm(r1 - r0, m - r0, bk, -1.f, mapPt[kb & 1], 0, r0, mapPt[kb & 1], 0, r0, 1.f, Ct,
                                     n, 1, nullptr, 0, split3, umma_err, s);
                });
        }
        return timed(kBlkTrailingUpdate, gemm_flops(r1 - r0, m - r0, bk, 1), s, [&] {
            return gemm<T, Tacc, T, true, false>(r1 - r0, m - r0, bk, Tacc(-1), pb + r0, m, pb + r0, m, Tacc(1), Ct, n,
                                                 1, part, part_elems, s);
        });
    };
    SideStream* side = side_stream();
    if (!side) return CHOL_ERR_CUDA;
    std::lock_guard<std::mutex> side_lock(side->mu);
    if (panel(0, s, part, part_elems) != cudaSuccess) return CHOL_ERR_CUDA;
    for (int kb = 0; kb + 1 < nb; ++kb) {
        const int k0 = kb * b;
        const int bk = std::min(b, n - k0);
        const int m = n - k0 - bk;
        const int bn = std::min(b, m);  // rows of block kb+1
        if (update(kb, 0, bn) != cudaSuccess) return CHOL_ERR_CUDA;
        if (cudaEventRecord(side->ready, s) != cudaSuccess) return CHOL_ERR_CUDA;
        if (cudaStreamWaitEvent(side->s, side->ready, 0) != cudaSuccess) return CHOL_ERR_CUDA;
        if (panel(kb + 1, side->s, part2, part2_elems) != cudaSuccess) return CHOL_ERR_CUDA;
        if (cudaEventRecord(side->done, side->s) != cudaSuccess) return CHOL_ERR_CUDA;
        if (update(kb, bn, m) != cudaSuccess) return CHOL_ERR_CUDA;
        if (cudaStreamWaitEvent(s, side->done, 0) != cudaSuccess) return CHOL_ERR_CUDA;
    }
    if (R) k_copy_upper<T><<<g1, 256, 0, s>>>(R, X, n, failed);
    if (!want_inv) return cudaGetLastError() == cudaSuccess ? CHOL_OK : CHOL_ERR_CUDA;
    // ---------------- inverse, block rows last..first
    for (int ib = nb - 1; ib >= 0; --ib) {
        const int i0 = ib * b;
        const int bi = std::min(b, n - i0);
        const int m = n - i0 - bi;
        const T* RinvI = Rinv + (size_t)ib * b * b;
        if (m > 0) {
            const T* RIr = X + (int64_t)i0 * n + i0 + bi;          // R_I,>I   (bi x m, ld n)
            const T* Xrr = X + (int64_t)(i0 + bi) * n + i0 + bi;  // X_>I,>I  (m x m, ld n, full)
            // P = R_I,>I X_>I,>I  (X is symmetric, so X_>I,>I read by rows is K-major)
            cudaError_t e;
            if (use_tc && bi == b) {
                e = timed(kBlkInverseProduct, gemm_flops(bi, m, m, 0), s, [&] {
                    return umma_gemm(bi, m, m, 1.f, mapX, i0 + bi, i0, mapX, i0 + bi, i0 + bi, 0.f,
                                     reinterpret_cast<float*>(P), m, 0, reinterpret_cast<float*>(part), part_elems,
                                     split3, umma_err, s);
                });
            } else {
                e = timed(kBlkInverseProduct, gemm_flops(bi, m, m, 0), s, [&] {
                    return gemm<T, Tacc, T, false, false>(bi, m, m, Tacc(1), RIr, n, Xrr, n, Tacc(0), P, m, 0, part,
                                                          part_elems, s);
                });
            }
            if (e != cudaSuccess) return CHOL_ERR_CUDA;
            // P2 = -R_II^{-1} P   (X_I,>I)
            e = gemm<T, Tacc, T, false, false>(bi, m, bi, Tacc(-1), RinvI, bi, P, m, Tacc(0), P2, m, 0, part,
                                              part_elems, s);
            if (e != cudaSuccess) return CHOL_ERR_CUDA;
            // Z = R_I,>I X_I,>I^T
            e = gemm<T, Tacc, T, false, true>(bi, bi, m, Tacc(1), RIr, n, P2, m, Tacc(0), Z, bi, 0, part, part_elems,
                                             s);
            if (e != cudaSuccess) return CHOL_ERR_CUDA;
            k_put_panel<T><<<g1, 256, 0, s>>>(X, n, i0, i0 + bi, bi, m, P2, 1, failed);
        }
        const int xt = (bi + kXdT - 1) / kXdT;
        k_blk_xdiag<T><<<dim3(xt, xt), 256, 0, s>>>(X, n, i0, bi, RinvI, m > 0 ? Z : nullptr, failed);
    }
    if (use_tc) k_report_umma<<<1, 1, 0, s>>>(umma_err, failed, err_word);
    k_nan_if_failed<T><<<g1, 256, 0, s>>>(X, (int64_t)n * n, failed);
    if (cudaGetLastError() != cudaSuccess) return CHOL_ERR_CUDA;

    // ---------------- refinement (FP32 only): X += X E, E = I - A X.  The
    // residual is formed transposed, E^T = I - X A (both are symmetric), so
    // that the correction's right operand is read by rows, K-major, as the
    // tensor cores take it.  X E = X - X A X is symmetric: only its upper half
    // is formed, and after each step the upper half of X is mirrored.
    if (refine_steps > 0 && sizeof(T) == 4) {
        float* Af = w.take<float>((size_t)n * n);
        double* E = w.take<double>((size_t)n * n);
        float* Et = w.take<float>((size_t)n * n);  // E^T, row-major
        const float* A32 = reinterpret_cast<const float*>(A);
        float* X32 = reinterpret_cast<float*>(X);
        k_sym_full<float><<<g1, 256, 0, s>>>(Af, A32, n);
        CUtensorMap mapE;
        const bool tc_corr = use_tc && make_map(&mapE, Et, n, n, n);
        for (int st = 0; st < refine_steps; ++st) {
            cudaError_t e;
            if (resid64) {
                // IEEE FP64 accumulation of the exact FP64 products of the FP32 values
                k_identity<double><<<g1, 256, 0, s>>>(E, n);
                e = timed(kBlkResidual, gemm_flops(n, n, n, 0), s, [&] {
                    return gemm<float, double, double, false, false>(n, n, n, -1.0, X32, n, Af, n, 1.0, E, n, 0,
                                                                     nullptr, 0, s);
                });
                if (e != cudaSuccess) return CHOL_ERR_CUDA;
                k_narrow<<<g1, 256, 0, s>>>(Et, E, (int64_t)n * n);
            } else {
                // compensated FP32 pairs (about 48 bits), no FP64 arithmetic
                e = timed(kBlkResidual, gemm_flops(n, n, n, 0), s, [&] {
                    const dim3 grid((n + GB_N - 1) / GB_N, (n + GB_M - 1) / GB_M);
                    k_resid_f2<<<grid, GB_THREADS, 0, s>>>(n, X32, Af, Et);
                    return cudaGetLastError();
                });
                if (e != cudaSuccess) return CHOL_ERR_CUDA;
            }
            // the correction X E goes to a separate buffer (the FP64 one, now free): the
            // product reads X while it runs.  On the tensor cores as split TF32 (FP32-level
            // accuracy on a term of relative size kappa u), else on the CUDA cores
            float* Cx = reinterpret_cast<float*>(E);
            e = timed(kBlkCorrection, gemm_flops(n, n, n, 1), s, [&] {
                if (tc_corr)
                    return umma_gemm(n, n, n, 1.f, mapX, 0, 0, mapE, 0, 0, 0.f, Cx, n, 1,
                                     reinterpret_cast<float*>(part), part_elems, 1, umma_err, s);
                return gemm<float, float, float, false, true>(n, n, n, 1.0f, X32, n, Et, n, 0.0f, Cx, n, 1, nullptr,
                                                              0, s);
            });
            if (e != cudaSuccess) return CHOL_ERR_CUDA;
            k_axpy<<<g1, 256, 0, s>>>(X32, Cx, (int64_t)n * n);
            // the upper half is the result (the lower half of Cx was not formed), mirrored in place
            k_sym_full<float><<<g1, 256, 0, s>>>(X32, X32, n);
        }
        if (tc_corr) k_report_umma<<<1, 1, 0, s>>>(umma_err, failed, err_word);
        if (cudaGetLastError() != cudaSuccess) return CHOL_ERR_CUDA;
    }
    return CHOL_OK;
}

// One complex Hermitian matrix through its real embedding (k_embed_hermitian):
// the real path of order 2n on M in the workspace, then X = P + iQ.  info is
// the embedding's (a row in 1..2n).
template <typename Rl>
static chol_status_t blocked_complex(const cpx<Rl>* A, cpx<Rl>* X, int n, int32_t* info, int pivot64,
                                     int refine_steps, int resid64, int tc, int* err_word, char* ws, cudaStream_t s) {
    const int n2 = 2 * n;
    const size_t mbytes = align256((size_t)n2 * n2 * sizeof(Rl));
    Rl* M = reinterpret_cast<Rl*>(ws);
    Rl* XM = reinterpret_cast<Rl*>(ws + mbytes);
    const int tiles = (n + kEmT - 1) / kEmT;
    k_embed_hermitian<Rl><<<dim3(tiles, tiles), dim3(kEmT, 8), 0, s>>>(A, M, n);
    if (cudaGetLastError() != cudaSuccess) return CHOL_ERR_CUDA;
    chol_status_t st;
    if constexpr (sizeof(Rl) == 4)
        st = blocked_one<float>(M, nullptr, XM, n2, info, pivot64, refine_steps, resid64, 1, tc, err_word,
                                ws + 2 * mbytes, s);
    else
        st = blocked_one<double>(M, nullptr, XM, n2, info, 0, 0, 0, 1, 0, err_word, ws + 2 * mbytes, s);
    if (st != CHOL_OK) return st;
    const int grid = std::max(1, std::min((int)(((int64_t)n * n + 255) / 256), device_info().sms * 8));
    k_extract_hermitian<Rl><<<grid, 256, 0, s>>>(XM, X, n);
    return cudaGetLastError() == cudaSuccess ? CHOL_OK : CHOL_ERR_CUDA;
}

chol_status_t blocked_run(int dtype, int32_t batch, int32_t n, const void* A, void* R, void* X, int32_t* info,
                          int pivot64, int refine_steps, int resid64, int want_inv, int tc, int* err_word, void* ws,
                          cudaStream_t s) {
    if ((dtype == CHOL_C64 || dtype == CHOL_C128) && (R != nullptr || !want_inv)) return CHOL_ERR_UNSUPPORTED;
    for (int32_t bi = 0; bi < batch; ++bi) {
        const int64_t o = (int64_t)bi * n * n;
        chol_status_t st = CHOL_OK;
        BlkTiming* tm = t_blk;
        cudaEvent_t w0 = tm ? tm->take() : nullptr, w1 = tm ? tm->take() : nullptr;
        if (w0 && w1 && cudaEventRecord(w0, s) != cudaSuccess) return CHOL_ERR_CUDA;
        if (dtype == CHOL_F32)
            st = blocked_one<float>(static_cast<const float*>(A) + o, R ? static_cast<float*>(R) + o : nullptr,
                                    static_cast<float*>(X) + o, n, info ? info + bi : nullptr, pivot64,
                                    refine_steps, resid64, want_inv, tc, err_word, static_cast<char*>(ws), s);
        else if (dtype == CHOL_F64)
            st = blocked_one<double>(static_cast<const double*>(A) + o, R ? static_cast<double*>(R) + o : nullptr,
                                     static_cast<double*>(X) + o, n, info ? info + bi : nullptr, 0, 0, 0, want_inv,
                                     0, err_word, static_cast<char*>(ws), s);
        else if (dtype == CHOL_C64)
            st = blocked_complex<float>(static_cast<const cpx<float>*>(A) + o, static_cast<cpx<float>*>(X) + o, n,
                                        info ? info + bi : nullptr, pivot64, refine_steps, resid64, tc, err_word,
                                        static_cast<char*>(ws), s);
        else if (dtype == CHOL_C128)
            st = blocked_complex<double>(static_cast<const cpx<double>*>(A) + o, static_cast<cpx<double>*>(X) + o,
                                         n, info ? info + bi : nullptr, 0, 0, 0, 0, err_word, static_cast<char*>(ws),
                                         s);
        else
            return CHOL_ERR_UNSUPPORTED;
        if (st != CHOL_OK) return st;
        if (w0 && w1) {
            if (cudaEventRecord(w1, s) != cudaSuccess) return CHOL_ERR_CUDA;
            tm->ev[kBlkWholeCall].push_back({w0, w1});
            tm->flops[kBlkWholeCall] += (double)n * n * n;  // the factor's n^3/3 and the inverse's 2 n^3/3
        }
    }
    return CHOL_OK;
}

}  // namespace cholinv
