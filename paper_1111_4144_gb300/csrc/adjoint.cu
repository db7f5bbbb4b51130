// Adjoint of the inverse on Hermitian matrices (not in the paper):
//   dA = -X S X,   S = (G + G^H) / 2,
// the gradient of a real loss L(X) with respect to a Hermitian A when
// X = A^{-1} and G = dL/dX.  It reuses the forward X (no refactorisation).
//
// Orders up to 32: a register-tiled warp per matrix (k_backward_tiled).
// Larger orders (and complex128): one warp per matrix with X (expanded from
// its stored upper half) and S as squares in shared memory; T = S X is
// formed column by column (lane j owns columns j and j+32), then the upper
// half of -X T, mirrored to keep dA exactly Hermitian.
#include <algorithm>
#include <mutex>
#include <type_traits>

#include "batched.cuh"
#include "tile.cuh"
#include "dispatch.h"

namespace cholinv {

template <typename V>
CHOL_HD size_t bwd_warp_bytes(int N) {
    const size_t b = (size_t)3 * N * (N + 1) * sizeof(V);
    return (b + 15) / 16 * 16;
}

template <typename V>
__global__ void k_backward(BwdParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = p.max_n;
    const int LD = N + 1;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, wpc = blockDim.x >> 5;
    V* Xf = reinterpret_cast<V*>(smem_raw + (size_t)w * bwd_warp_bytes<V>(N));
    V* Sf = Xf + (size_t)N * LD;
    V* Tf = Sf + (size_t)N * LD;
    const V* X = static_cast<const V*>(p.X);
    const V* G = static_cast<const V*>(p.G);
    V* dA = static_cast<V*>(p.dA);

    for (int b = blockIdx.x * wpc + w; b < p.batch; b += gridDim.x * wpc) {
        const int n = p.n ? p.n[b] : N;
        if (n <= 0 || n > N) continue;
        const int64_t og = p.off ? p.off[b] : (int64_t)b * N * N;
        const int64_t ox = p.xoff ? p.xoff[b] : (int64_t)b * (p.layout ? tri64(N) : (int64_t)N * N);
        __syncwarp();  // the previous matrix's squares are no longer read
        stage_hermitian(X + ox, n, p.layout, Xf, LD, lane);
        // G into Tf (free until T = S X), then S = (G + G^H)/2 into Sf
        warp_rows<false>(G + og, n, n, 0, lane, [&](int i, int j, V v) { Tf[i * LD + j] = v; });
        __syncwarp();
        for (int i = 0; i < n; ++i)
            for (int j = i + lane; j < n; j += 32) {
                using R = typename traits<V>::real;
                const V sij = scale_v(Tf[i * LD + j] + conj_v(Tf[j * LD + i]), R(0.5));
                Sf[i * LD + j] = (i == j) ? from_real<V>(re_of(sij)) : sij;
                Sf[j * LD + i] = conj_v(sij);
            }
        __syncwarp();
        // T = S X
        for (int j = lane; j < n; j += 32)
            for (int i = 0; i < n; ++i) {
                V acc = zero_v<V>();
                for (int k = 0; k < n; ++k) acc = fma_v(Sf[i * LD + k], Xf[k * LD + j], acc);
                Tf[i * LD + j] = acc;
            }
        __syncwarp();
        // dA = -X T (upper half computed, mirrored)
        for (int j = lane; j < n; j += 32)
            for (int i = 0; i <= j; ++i) {
                V acc = zero_v<V>();
                for (int k = 0; k < n; ++k) acc = fma_v(Xf[i * LD + k], Tf[k * LD + j], acc);
                V d = zero_v<V>() - acc;
                if (i == j) d = from_real<V>(re_of(d));
                if (p.flags & CHOL_FLAG_GRAD_UPPER) {
                    using R = typename traits<V>::real;
                    dA[og + (int64_t)i * n + j] = (i == j) ? d : scale_v(d, R(2));
                    if (i != j) dA[og + (int64_t)j * n + i] = zero_v<V>();
                } else {
                    dA[og + (int64_t)i * n + j] = d;
                    if (i != j) dA[og + (int64_t)j * n + i] = conj_v(d);
                }
            }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Register-tiled form for orders up to 32 (zero-padded to 32): one warp per
// matrix, lane l computes the 4 x 8 block at rows 4 (l / 4).., columns
// 8 (l % 4).. of each 32 x 32 product, from shared-memory row slices (a
// 4-wide slice of the left operand, stored transposed, and an 8-wide slice
// of the right one per k).
//   Xs: X in full (Xs[k][r] = x_kr), the right operand of T = S X and,
//       conjugated, the transposed left operand of X T;
//   St: S^T (St[k][r] = s_rk), S = (G + G^H)/2, G first staged in Ts;
//   Ts: T = S X; then -X T is staged in St and its upper half written,
//       mirrored, so that dA is exactly Hermitian.
// ---------------------------------------------------------------------------

template <typename V>
CHOL_HD size_t bwd_tiled_warp_bytes() {
    return (size_t)3 * kTB * kTLD * sizeof(V);
}


template <typename V>
__global__ void __launch_bounds__(128) k_backward_tiled(BwdParams p) {
    using R = typename traits<V>::real;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, wpc = blockDim.x >> 5;
    V* Xs = reinterpret_cast<V*>(smem_raw + (size_t)w * bwd_tiled_warp_bytes<V>());
    V* St = Xs + kTB * kTLD;
    V* Ts = St + kTB * kTLD;
    const V* X = static_cast<const V*>(p.X);
    const V* G = static_cast<const V*>(p.G);
    V* dA = static_cast<V*>(p.dA);
    const int r0 = (lane / 4) * 4, c0 = (lane % 4) * 8;
    const int N = p.max_n;
    for (int b = blockIdx.x * wpc + w; b < p.batch; b += gridDim.x * wpc) {
        const int n = p.n ? p.n[b] : N;
        if (n <= 0 || n > N) continue;
        const int64_t og = p.off ? p.off[b] : (int64_t)b * N * N;
        const int64_t ox = p.xoff ? p.xoff[b] : (int64_t)b * (p.layout ? tri64(N) : (int64_t)N * N);
        __syncwarp();  // the previous matrix's squares are no longer read
        if (n < kTB) {
            // the zero padding rows and columns n..kTB-1 (the products run over kTB)
            for (int i = 0; i < kTB; ++i)
                if (i >= n || lane >= n) Xs[i * kTLD + lane] = St[i * kTLD + lane] = zero_v<V>();
        }
        // G staged in Ts; X in full from its upper half (lanes over columns)
        constexpr int U = sizeof(V) == 4 ? 16 : 8;  // rows a round: the loads in flight per lane
        warp_rows<false, 1, U>(G + og, n, n, 0, lane, [&](int i, int j, V v) { Ts[i * kTLD + j] = v; });
        warp_rows<true, 1, U>(X + ox, n, n, p.layout, lane, [&](int i, int j, V v) {
            const V x = (i == j) ? from_real<V>(re_of(v)) : v;
            Xs[i * kTLD + j] = x;
            Xs[j * kTLD + i] = conj_v(x);
        });
        __syncwarp();
        // St[k][r] = s_rk = (g_rk + conj(g_kr)) / 2, lanes over k
        if (lane < n) {
            for (int r = 0; r < n; ++r) {
                const int k = lane;
                V sv = scale_v(Ts[r * kTLD + k] + conj_v(Ts[k * kTLD + r]), R(0.5));
                if (k == r) sv = from_real<V>(re_of(sv));
                St[k * kTLD + r] = sv;
            }
        }
        __syncwarp();
        V acc[4][8];
        // T = S X
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[r][c] = zero_v<V>();
        tile_product<V, false>(St, Xs, r0, c0, acc);
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 8; ++c) Ts[(r0 + r) * kTLD + c0 + c] = acc[r][c];
        __syncwarp();
        // X T: the transposed left operand is conj(X) (X Hermitian): conj(Xs[k][r]) = x_rk
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[r][c] = zero_v<V>();
        tile_product<V, traits<V>::cplx>(Xs, Ts, r0, c0, acc);
        // -X T staged in St (S is no longer read), then dA row by row
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 8; ++c) St[(r0 + r) * kTLD + c0 + c] = zero_v<V>() - acc[r][c];
        __syncwarp();
        const bool upper_param = (p.flags & CHOL_FLAG_GRAD_UPPER) != 0;
        if (lane < n) {
            for (int i = 0; i < n; ++i) {
                const int j = lane;
                V d = (i <= j) ? St[i * kTLD + j] : conj_v(St[j * kTLD + i]);
                if (i == j) d = from_real<V>(re_of(d));
                if (upper_param) d = (i < j) ? scale_v(d, R(2)) : (i == j) ? d : zero_v<V>();
                dA[og + i * n + j] = d;
            }
        }
        __syncwarp();
    }
}

template <typename V>
static cudaError_t launch_bwd_tiled(const BwdParams& p, cudaStream_t s, bool dry) {
    static std::once_flag once;
    static cudaError_t setup = cudaSuccess;
    constexpr int warps = 4;
    const size_t smem = bwd_tiled_warp_bytes<V>() * warps;
    std::call_once(once, [&] {
        setup = cudaFuncSetAttribute(k_backward_tiled<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
    if (setup != cudaSuccess || dry) return setup;
    int per_sm = 1;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_backward_tiled<V>, 32 * warps, smem);
    if (e != cudaSuccess) return e;
    const int grid = std::max(1, std::min((p.batch + warps - 1) / warps, device_info().sms * std::max(per_sm, 1)));
    k_backward_tiled<V><<<grid, 32 * warps, smem, s>>>(p);
    return cudaGetLastError();
}

template <typename V>
static cudaError_t launch_bwd_t(const BwdParams& p, cudaStream_t s, bool dry) {
    // orders up to 32 (complex128 excepted: its register tile is too large)
    if constexpr (!std::is_same<V, cpx<double>>::value)
        if (p.max_n <= kTB) return launch_bwd_tiled<V>(p, s, dry);
    static std::once_flag once;
    static cudaError_t setup = cudaSuccess;
    std::call_once(once, [&] {
        setup = cudaFuncSetAttribute(k_backward<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    });
    if (setup != cudaSuccess || dry) return setup;
    const size_t per = bwd_warp_bytes<V>(p.max_n);
    const int warps = (int)std::max<size_t>(1, std::min<size_t>(4, 98304 / per));
    int per_sm = 1;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_backward<V>, 32 * warps, per * warps);
    if (e != cudaSuccess) return e;
    const int grid = std::max(1, std::min((p.batch + warps - 1) / warps, device_info().sms * std::max(per_sm, 1)));
    k_backward<V><<<grid, 32 * warps, per * warps, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_backward(int dtype, const BwdParams& p, cudaStream_t s, bool dry) {
    switch (dtype) {
        case CHOL_F32: return launch_bwd_t<float>(p, s, dry);
        case CHOL_F64: return launch_bwd_t<double>(p, s, dry);
        case CHOL_C64: return launch_bwd_t<cpx<float>>(p, s, dry);
        case CHOL_C128: return launch_bwd_t<cpx<double>>(p, s, dry);
    }
    return cudaErrorInvalidValue;
}

}  // namespace cholinv
