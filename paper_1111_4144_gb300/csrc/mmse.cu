// MMSE filters W = (H^* H + s2 I)^{-1} H^* of a batch of channel matrices H
// (chol_mmse_batched; the Hermitian inverse by Sec. II + Sec. IV.A, the
// usual consumer of the MIMO covariances).  With s2 = 0 and a square H = D^*
// it gives W = (D D^*)^{-1} D, whose conjugate transpose is the inverse of
// the non-Hermitian D in Sec. III.C's form, D^{-1} = D^* (D D^*)^{-1}.
//
// Three steps on the caller's stream:
//   k_gram   A = H^* H + s2 I, packed upper, one warp per matrix (H staged
//            in shared memory, lanes over the entries of A's triangle);
//   the batched inverse of A (the size-class kernels of chol_inv_batched);
//   k_apply  W = X H^*, X the full Hermitian inverse (its upper half
//            mirrored in shared memory), lanes over the entries of W.
// Orders up to 16 with up to 32 rows take register-tiled forms of the two
// products (k_gram16, k_apply16).
#include <algorithm>
#include <mutex>
#include <type_traits>

#include "batched.cuh"
#include "dispatch.h"

namespace cholinv {

// shared memory of one warp: H (k_gram) or H^T with rows of m + 1 (k_apply), and X
template <typename V>
CHOL_HD size_t mmse_warp_elems(int max_n, int max_m) {
    return (size_t)(max_m + 1) * max_n + (size_t)max_n * (max_n + 1);
}

// Order and rows of matrix b, and its offsets in H, W and the packed A / X.
CHOL_D void mmse_geom(const MmseParams& p, int64_t b, int& n, int& m, int64_t& oh, int64_t& ow, int64_t& oa) {
    n = p.n ? p.n[b] : p.max_n;
    m = p.m ? p.m[b] : p.max_m;
    oh = p.hoff ? p.hoff[b] : b * (int64_t)p.max_m * p.max_n;
    ow = p.woff ? p.woff[b] : b * (int64_t)p.max_n * p.max_m;
    oa = b * tri64(p.max_n);
}

template <typename V>
__global__ void k_gram(MmseParams p, typename traits<V>::real s2) {
    using R = typename traits<V>::real;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, wpc = blockDim.x >> 5;
    V* Hs = reinterpret_cast<V*>(smem_raw) + (size_t)w * mmse_warp_elems<V>(p.max_n, p.max_m);
    const V* H = static_cast<const V*>(p.H);
    V* A = static_cast<V*>(p.A);
    for (int64_t b = (int64_t)blockIdx.x * wpc + w; b < p.batch; b += (int64_t)gridDim.x * wpc) {
        int n, m;
        int64_t oh, ow, oa;
        mmse_geom(p, b, n, m, oh, ow, oa);
        if (n < 1 || n > p.max_n || m < 0 || m > p.max_m) continue;  // invalid orders are flagged by the inverse
        __syncwarp();  // the previous matrix's H is no longer read
        warp_gather(H + oh, m * n, lane, [&](int e, V v) { Hs[e] = v; });
        __syncwarp();
        const int T = tri(n);
        for (int e = lane; e < T; e += 32) {
            int i, j;
            tri_rc(n, e, i, j);
            // a_ij = sum_r conj(h_ri) h_rj (+ s2 on the diagonal)
            V acc = zero_v<V>();
            for (int r = 0; r < m; ++r) acc = fma_v(conj_v(Hs[r * n + i]), Hs[r * n + j], acc);
            if (i == j) acc = from_real<V>(re_of(acc) + s2);
            A[oa + e] = acc;
        }
        __syncwarp();
    }
}

template <typename V>
__global__ void k_apply(MmseParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, wpc = blockDim.x >> 5;
    V* Ht = reinterpret_cast<V*>(smem_raw) + (size_t)w * mmse_warp_elems<V>(p.max_n, p.max_m);  // H^T
    V* Xs = Ht + (size_t)(p.max_m + 1) * p.max_n;
    const V* H = static_cast<const V*>(p.H);
    const V* X = static_cast<const V*>(p.X);
    V* W = static_cast<V*>(p.W);
    for (int64_t b = (int64_t)blockIdx.x * wpc + w; b < p.batch; b += (int64_t)gridDim.x * wpc) {
        int n, m;
        int64_t oh, ow, oa;
        mmse_geom(p, b, n, m, oh, ow, oa);
        if (n < 1 || n > p.max_n || m < 0 || m > p.max_m) continue;
        const bool bad = p.info && p.info[b] != 0;
        __syncwarp();  // the previous matrix's H and X are no longer read
        // H transposed (row stride m + 1), so that lanes over k read consecutive words below
        warp_gather(H + oh, m * n, lane, [&](int e, V v) {
            const int r = e / n, c = e - r * n;
            Ht[c * (m + 1) + r] = v;
        });
        const int LD = n + 1;
        warp_gather(X + oa, tri(n), lane, [&](int e, V x) {
            int i, j;
            tri_rc(n, e, i, j);
            Xs[i * LD + j] = x;
            Xs[j * LD + i] = conj_v(x);
        });
        __syncwarp();
        // w_ik = sum_j x_ij conj(h_kj), W row-major n x m
        for (int e = lane; e < n * m; e += 32) {
            const int i = e / m, k = e - i * m;
            V acc = zero_v<V>();
            for (int j = 0; j < n; ++j) acc = fma_conjb(Xs[i * LD + j], Ht[j * (m + 1) + k], acc);
            W[ow + e] = bad ? nan_v<V>() : acc;
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Register-tiled forms for orders up to 16 with up to 32 rows (the MIMO
// shapes): one warp per matrix, lane l holding a 2-row block of the product
// (rows 2 (l / 4)..), so that each shared-memory load feeds several
// multiply-adds instead of one.
// ---------------------------------------------------------------------------
constexpr int kMN = 16;        // orders
constexpr int kMM = 32;        // rows of H
constexpr int kGLD = kMN + 4;  // row stride of H in k_gram16 and of X in k_apply16
// row stride of H^* (transposed) in k_apply16: odd, so that the transposing
// stores of a warp's consecutive elements land on distinct banks
constexpr int kALD = kMM + 1;

// acc += a b (complex64 on paired FP32 instructions: the two parts of an entry)
template <typename V>
CHOL_D void mac(V& acc, V a, V b) {
    if constexpr (std::is_same<V, cpx<float>>::value) {
        float2 q = make_float2(acc.re, acc.im);
        q = __ffma2_rn(make_float2(a.re, a.re), make_float2(b.re, b.im), q);
        q = __ffma2_rn(make_float2(a.im, a.im), make_float2(-b.im, b.re), q);
        acc = {q.x, q.y};
    } else {
        acc = fma_v(a, b, acc);
    }
}

template <typename V>
CHOL_HD size_t mmse16_warp_elems() {
    return (size_t)kMN * kALD + (size_t)kMN * kGLD;  // the larger of the two kernels' needs
}

// A = H^* H + s2 I: lane l computes a_ij for i = 2 (l / 4) + {0, 1},
// j = 4 (l % 4) + {0..3}, as sum_k conj(h_ki) h_kj over H's m rows.
template <typename V>
__global__ void __launch_bounds__(256) k_gram16(MmseParams p, typename traits<V>::real s2) {
    using R = typename traits<V>::real;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, wpc = blockDim.x >> 5;
    V* Hs = reinterpret_cast<V*>(smem_raw) + (size_t)w * mmse16_warp_elems<V>();  // [m][kGLD]
    const V* H = static_cast<const V*>(p.H);
    V* A = static_cast<V*>(p.A);
    const int r0 = (lane / 4) * 2, c0 = (lane % 4) * 4;
    for (int64_t b = (int64_t)blockIdx.x * wpc + w; b < p.batch; b += (int64_t)gridDim.x * wpc) {
        int n, m;
        int64_t oh, ow, oa;
        mmse_geom(p, b, n, m, oh, ow, oa);
        if (n < 1 || n > p.max_n || m < 0 || m > p.max_m) continue;  // invalid orders are flagged by the inverse
        __syncwarp();  // the previous matrix's H is no longer read
        warp_gather(H + oh, m * n, lane, [&](int e, V v) {
            const int k = e / n, c = e - k * n;
            Hs[k * kGLD + c] = v;
        });
        __syncwarp();
        V acc[2][4];
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] = zero_v<V>();
#pragma unroll 4
        for (int k = 0; k < m; ++k) {
            V a[2], bb[4];
#pragma unroll
            for (int r = 0; r < 2; ++r) a[r] = conj_v(Hs[k * kGLD + r0 + r]);
#pragma unroll
            for (int c = 0; c < 4; ++c) bb[c] = Hs[k * kGLD + c0 + c];
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) mac(acc[r][c], a[r], bb[c]);
        }
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int i = r0 + r, j = c0 + c;
                if (i <= j && j < n) A[oa + pidx(n, i, j)] = (i == j) ? from_real<V>(re_of(acc[r][c]) + s2) : acc[r][c];
            }
    }
}

// W = X H^*: lane l computes w_ik for i = 2 (l / 4) + {0, 1},
// k = 8 (l % 4) + {0..7}, as sum_j x_ij conj(h_kj) over the n columns.
template <typename V>
__global__ void __launch_bounds__(256) k_apply16(MmseParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, wpc = blockDim.x >> 5;
    V* Hc = reinterpret_cast<V*>(smem_raw) + (size_t)w * mmse16_warp_elems<V>();  // [n][kALD]: conj(h_kj) at [j][k]
    V* Xs = Hc + kMN * kALD;                                                       // [n][kGLD]: x_ji at [j][i]
    const V* H = static_cast<const V*>(p.H);
    const V* X = static_cast<const V*>(p.X);
    V* W = static_cast<V*>(p.W);
    const int r0 = (lane / 4) * 2, c0 = (lane % 4) * 8;
    for (int64_t b = (int64_t)blockIdx.x * wpc + w; b < p.batch; b += (int64_t)gridDim.x * wpc) {
        int n, m;
        int64_t oh, ow, oa;
        mmse_geom(p, b, n, m, oh, ow, oa);
        if (n < 1 || n > p.max_n || m < 0 || m > p.max_m) continue;
        const bool bad = p.info && p.info[b] != 0;
        __syncwarp();  // the previous matrix's H and X are no longer read
        warp_gather(H + oh, m * n, lane, [&](int e, V v) {
            const int k = e / n, j = e - k * n;
            Hc[j * kALD + k] = conj_v(v);
        });
        warp_gather(X + oa, tri(n), lane, [&](int e, V x) {
            int i, j;
            tri_rc(n, e, i, j);
            Xs[i * kGLD + j] = x;
            Xs[j * kGLD + i] = conj_v(x);
        });
        __syncwarp();
        V acc[2][8];
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[r][c] = zero_v<V>();
#pragma unroll 4
        for (int j = 0; j < n; ++j) {
            V a[2], bb[8];
#pragma unroll
            for (int r = 0; r < 2; ++r) a[r] = conj_v(Xs[j * kGLD + r0 + r]);  // x_ij = conj(x_ji)
#pragma unroll
            for (int c = 0; c < 8; ++c) bb[c] = Hc[j * kALD + c0 + c];
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int c = 0; c < 8; ++c) mac(acc[r][c], a[r], bb[c]);
        }
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int i = r0 + r, k = c0 + c;
                if (i < n && k < m) W[ow + (int64_t)i * m + k] = bad ? nan_v<V>() : acc[r][c];
            }
    }
}

template <typename V>
static cudaError_t launch_mmse_t(int stage, const MmseParams& p, double s2, cudaStream_t s, bool dry) {
    using R = typename traits<V>::real;
    static std::once_flag once;
    static cudaError_t setup = cudaSuccess;
    std::call_once(once, [&] {
        setup = cudaFuncSetAttribute(k_gram<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (setup == cudaSuccess)
            setup = cudaFuncSetAttribute(k_apply<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (setup == cudaSuccess)
            setup = cudaFuncSetAttribute(k_gram16<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (setup == cudaSuccess)
            setup = cudaFuncSetAttribute(k_apply16<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    });
    if (setup != cudaSuccess || dry) return setup;
    if (p.max_n <= kMN && p.max_m <= kMM) {
        // the register-tiled forms, eight warps (matrices) per CTA
        constexpr int warps = 8;
        const size_t smem = mmse16_warp_elems<V>() * sizeof(V) * warps;
        const int grid = std::max(1, std::min((p.batch + warps - 1) / warps, device_info().sms * 8));
        if (stage == 0)
            k_gram16<V><<<grid, 32 * warps, smem, s>>>(p, (R)s2);
        else
            k_apply16<V><<<grid, 32 * warps, smem, s>>>(p);
        return cudaGetLastError();
    }
    const size_t per = mmse_warp_elems<V>(p.max_n, p.max_m) * sizeof(V);
    const int warps = (int)std::max<size_t>(1, std::min<size_t>(8, 98304 / per));
    const int grid = std::max(1, std::min((p.batch + warps - 1) / warps, device_info().sms * 8));
    if (stage == 0)
        k_gram<V><<<grid, 32 * warps, per * warps, s>>>(p, (R)s2);
    else
        k_apply<V><<<grid, 32 * warps, per * warps, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_mmse(int dtype, int stage, const MmseParams& p, double s2, cudaStream_t s, bool dry) {
    switch (dtype) {
        case CHOL_F32: return launch_mmse_t<float>(stage, p, s2, s, dry);
        case CHOL_F64: return launch_mmse_t<double>(stage, p, s2, s, dry);
        case CHOL_C64: return launch_mmse_t<cpx<float>>(stage, p, s2, s, dry);
        case CHOL_C128: return launch_mmse_t<cpx<double>>(stage, p, s2, s, dry);
    }
    return cudaErrorInvalidValue;
}

}  // namespace cholinv
