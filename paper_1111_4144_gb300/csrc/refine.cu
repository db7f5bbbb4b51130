// Iterative refinement of a single-precision inverse (FP32 / complex64):
//   E  = I - A X        (residual: each product of two FP32 numbers exact,
//                        the sums accumulated in compensated FP32 pairs
//                        (about 48 bits) or, with CHOL_FLAG_RESIDUAL_FP64,
//                        in FP64)
//   X <- X + X E        (Newton-Schulz correction, FP32, upper half of X)
// The paper states the method's accuracy only for well-conditioned inputs
// (Sec. II); refinement recovers what FP32 arithmetic loses on harder ones.
//
// One warp per matrix.  A and the current X are expanded to full Hermitian
// squares in shared memory (global memory holds only their upper
// triangles).  For each column j, lanes (one per row) form column j of E in
// FP64 and park it in shared memory; then the lanes owning rows i <= j add
// row i of X times that column and write the new x_ij to global memory.
// The old X stays in shared memory until the step ends.
#include <algorithm>
#include <mutex>

#include "batched.cuh"
#include "dispatch.h"
#include "tile.cuh"

namespace cholinv {

template <typename V>
struct wide;  // the FP64 counterpart of a single-precision value type
template <> struct wide<float> { using type = double; };
template <> struct wide<cpx<float>> { using type = cpx<double>; };

CHOL_D double widen(float v) { return (double)v; }
CHOL_D cpx<double> widen(cpx<float> v) { return {(double)v.re, (double)v.im}; }
CHOL_D float narrow(double v) { return (float)v; }
CHOL_D cpx<float> narrow(cpx<double> v) { return {(float)v.re, (float)v.im}; }

// gamma = max_i a_ii x_ii lies in [1, (1 + kappa)^2 / (4 kappa)], kappa =
// kappa_2(A), for a Hermitian positive definite A: a_ii x_ii is
// (e_i^* A e_i)(e_i^* A^{-1} e_i), at least 1 by Cauchy-Schwarz and at most
// the Kantorovich bound.  The automatic mode refines a matrix once when gamma
// exceeds this threshold (reachable for kappa above about 16,382).
constexpr double kAutoRefineGamma = 4096.0;

template <typename V>
CHOL_HD size_t refine_warp_bytes(int N) {
    using W = typename wide<V>::type;
    const size_t b = (size_t)2 * N * (N + 1) * sizeof(V) + (size_t)N * sizeof(W);
    return (b + 15) / 16 * 16;
}

// Entry (i, j) of E = I - A X from row i of A and column j of X (shared
// memory, leading dimension LD): FP64 accumulation (R64), or compensated
// FP32 pairs (f2acc), rounded to FP32 at the end.
template <typename V, bool R64>
CHOL_D V resid_entry(const V* Arow, const V* Xcol, int LD, int n, bool diag) {
    if constexpr (R64) {
        using W = typename wide<V>::type;
        W acc = zero_v<W>();
        for (int k = 0; k < n; ++k) acc = fma_v(widen(Arow[k]), widen(Xcol[(size_t)k * LD]), acc);
        return narrow(diag ? from_real<W>(1.0) - acc : zero_v<W>() - acc);
    } else if constexpr (traits<V>::cplx) {
        f2acc re = f2_init(diag ? 1.f : 0.f), im = f2_init(0.f);
        for (int k = 0; k < n; ++k) {
            const V a = Arow[k], x = Xcol[(size_t)k * LD];
            f2_fma(re, -a.re, x.re);
            f2_fma(re, a.im, x.im);
            f2_fma(im, -a.re, x.im);
            f2_fma(im, -a.im, x.re);
        }
        return V{f2_value(re), f2_value(im)};
    } else {
        f2acc r = f2_init(diag ? 1.f : 0.f);
        for (int k = 0; k < n; ++k) f2_fma(r, -Arow[k], Xcol[(size_t)k * LD]);
        return f2_value(r);
    }
}

template <typename V, bool R64>
__global__ void k_refine(BatchParams p, int steps, int automatic) {
    using W = typename wide<V>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = p.max_n;
    const int LD = N + 1;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, wpc = blockDim.x >> 5;
    unsigned char* base = smem_raw + (size_t)w * refine_warp_bytes<V>(N);
    V* Af = reinterpret_cast<V*>(base);
    V* Xf = Af + (size_t)N * LD;
    V* ec = reinterpret_cast<V*>(Xf + (size_t)N * LD);  // column j of E
    const V* A = static_cast<const V*>(p.A);
    V* X = static_cast<V*>(p.X);

    for (int b = blockIdx.x * wpc + w; b < p.batch; b += gridDim.x * wpc) {
        const int n = p.n ? p.n[b] : N;
        if (n <= 0 || n > N) continue;
        if (p.info && p.info[b] != 0) continue;
        const int64_t o = p.off ? p.off[b] : (int64_t)b * (p.layout ? tri64(N) : (int64_t)N * N);
        auto gidx = [&](int i, int j) { return p.layout ? (int64_t)pidx(n, i, j) : (int64_t)i * n + j; };
        __syncwarp();  // the previous matrix's squares are no longer read
        stage_hermitian(A + o, n, p.layout, Af, LD, lane);
        int todo = steps;
        for (int s = 0; s <= todo; ++s) {
            // (re)load the current X (the columns below update it in memory)
            __syncwarp();
            stage_hermitian(static_cast<const V*>(X) + o, n, p.layout, Xf, LD, lane);
            __syncwarp();
            if (s == 0 && automatic) {
                double g = 0.0;
                for (int i = lane; i < n; i += 32)
                    g = fmax(g, (double)re_of(Af[i * LD + i]) * (double)re_of(Xf[i * LD + i]));
                for (int d = 16; d > 0; d >>= 1) g = fmax(g, __shfl_xor_sync(0xffffffffu, g, d));
                todo = g > kAutoRefineGamma ? 1 : 0;
            }
            if (s == todo) break;
            for (int j = 0; j < n; ++j) {
                for (int i = lane; i < n; i += 32) ec[i] = resid_entry<V, R64>(Af + i * LD, Xf + j, LD, n, i == j);
                __syncwarp();
                for (int i = lane; i <= j; i += 32) {
                    V acc = Xf[i * LD + j];
                    for (int k = 0; k < n; ++k) acc = fma_v(Xf[i * LD + k], ec[k], acc);
                    if (i == j) acc = from_real<V>(re_of(acc));
                    X[o + gidx(i, j)] = acc;
                }
                __syncwarp();
            }
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Register-tiled form for orders up to 32, compensated FP32 residual: one
// warp per matrix, the matrix zero-padded to a square of order TB (16 for
// orders up to 16, else 32); lane l holds the TR x TC block (4 x 8 or
// 2 x 4) at rows TR (l / 4).., columns TC (l % 4).. of E = I - A X
// (compensated pairs, two entries or the two parts of a complex entry per
// paired FP32 instruction) and then of the correction X E (plain FP32).
// A, X and E are full squares in shared memory (row stride TB + 4); the
// left operands' row slices come from their conjugate-transposed rows (both
// are Hermitian).
// ---------------------------------------------------------------------------
// A, X and E as padded squares, then the next matrix's A and X as stored
// (dense or packed), filled by asynchronous copies during this one's steps.
template <typename V, int TB>
CHOL_HD size_t refine_tiled_warp_bytes() {
    return (size_t)3 * TB * Tile<TB>::LD * sizeof(V) + (size_t)2 * TB * TB * sizeof(V);
}

// acc += a b with a, b real (paired lanes: two entries of a row) or complex
// (paired lanes: the real and imaginary parts of one entry), over a TR x TC block
template <typename V, int TR, int TC>
struct ResidTile;
template <int TR, int TC>
struct ResidTile<float, TR, TC> {
    f2acc2 acc[TR][TC / 2];  // [row][column pair]
    CHOL_D void init(int r0, int c0) {
#pragma unroll
        for (int r = 0; r < TR; ++r)
#pragma unroll
            for (int cp = 0; cp < TC / 2; ++cp) {
                const int i = r0 + r, j = c0 + 2 * cp;
                acc[r][cp].s = make_float2(i == j ? 1.f : 0.f, i == j + 1 ? 1.f : 0.f);
                acc[r][cp].c = make_float2(0.f, 0.f);
            }
    }
    // acc[r][c] -= a_r b_c over one k
    CHOL_D void step(const float (&a)[TR], const float (&b)[TC]) {
#pragma unroll
        for (int r = 0; r < TR; ++r)
#pragma unroll
            for (int cp = 0; cp < TC / 2; ++cp)
                f2_fma2(acc[r][cp], make_float2(-a[r], -a[r]), make_float2(b[2 * cp], b[2 * cp + 1]));
    }
    CHOL_D float value(int r, int c) const {
        const f2acc2& q = acc[r][c / 2];
        return (c & 1) ? __fadd_rn(q.s.y, q.c.y) : __fadd_rn(q.s.x, q.c.x);
    }
};
template <int TR, int TC>
struct ResidTile<cpx<float>, TR, TC> {
    f2acc2 acc[TR][TC];  // lanes x, y: real and imaginary parts
    CHOL_D void init(int r0, int c0) {
#pragma unroll
        for (int r = 0; r < TR; ++r)
#pragma unroll
            for (int c = 0; c < TC; ++c) {
                acc[r][c].s = make_float2(r0 + r == c0 + c ? 1.f : 0.f, 0.f);
                acc[r][c].c = make_float2(0.f, 0.f);
            }
    }
    // (a b).re = a.re b.re - a.im b.im, (a b).im = a.re b.im + a.im b.re; subtracted
    CHOL_D void step(const cpx<float> (&a)[TR], const cpx<float> (&b)[TC]) {
#pragma unroll
        for (int r = 0; r < TR; ++r)
#pragma unroll
            for (int c = 0; c < TC; ++c) {
                f2_fma2(acc[r][c], make_float2(-a[r].re, -a[r].re), make_float2(b[c].re, b[c].im));
                f2_fma2(acc[r][c], make_float2(a[r].im, -a[r].im), make_float2(b[c].im, b[c].re));
            }
    }
    CHOL_D cpx<float> value(int r, int c) const {
        const f2acc2& q = acc[r][c];
        return {__fadd_rn(q.s.x, q.c.x), __fadd_rn(q.s.y, q.c.y)};
    }
};

template <typename V, int TB>
__global__ void __launch_bounds__(128) k_refine_tiled(BatchParams p, int steps, int automatic) {
    constexpr int LD = Tile<TB>::LD, TR = Tile<TB>::TR, TC = Tile<TB>::TC;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = p.max_n;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, wpc = blockDim.x >> 5;
    V* As = reinterpret_cast<V*>(smem_raw + (size_t)w * refine_tiled_warp_bytes<V, TB>());
    V* Xs = As + TB * LD;
    V* Es = Xs + TB * LD;
    V* RawA = Es + TB * LD;
    V* RawX = RawA + TB * TB;
    const V* A = static_cast<const V*>(p.A);
    V* X = static_cast<V*>(p.X);
    const int r0 = (lane / 4) * TR, c0 = (lane % 4) * TC;
    // matrix b's order (0: nothing to refine) and element offset
    auto geom = [&](int b, int& n, int64_t& o) {
        n = p.n ? p.n[b] : N;
        if (n <= 0 || n > N || (p.info && p.info[b] != 0)) n = 0;
        o = p.off ? p.off[b] : (int64_t)b * (p.layout ? tri64(N) : (int64_t)N * N);
    };
    // matrix b's A and X as stored, into RawA / RawX (asynchronous)
    auto prefetch = [&](int b) {
        if (b < p.batch) {
            int n;
            int64_t o;
            geom(b, n, o);
            if (n > 0) {
                const int count = p.layout ? n * (n + 1) / 2 : n * n;
                warp_copy_async(RawA, A + o, count, lane);
                warp_copy_async(RawX, static_cast<const V*>(X) + o, count, lane);
            }
        }
        cp_async_commit();
    };
    const int stride = gridDim.x * wpc;
    int b = blockIdx.x * wpc + w;
    prefetch(b);
    for (; b < p.batch; b += stride) {
        int n;
        int64_t o;
        geom(b, n, o);
        cp_async_wait<0>();
        __syncwarp();  // every lane's copies are visible; the previous matrix's squares are no longer read
        if (n > 0) {
            if (n < TB) {
                // the zero padding rows and columns n..TB-1 (the products run over TB)
                for (int e = lane; e < TB * TB; e += 32) {
                    const int i = e / TB, j = e % TB;
                    if (i >= n || j >= n) As[i * LD + j] = Xs[i * LD + j] = zero_v<V>();
                }
            }
            unpack_hermitian(RawA, n, p.layout, As, LD, lane);
            unpack_hermitian(RawX, n, p.layout, Xs, LD, lane);
        }
        __syncwarp();  // the stored copies are read: the next matrix's may land there
        prefetch(b + stride);
        if (n == 0) continue;
        auto gidx = [&](int i, int j) { return p.layout ? (int64_t)pidx(n, i, j) : (int64_t)i * n + j; };
        int todo = steps;
#pragma unroll 1
        for (int s = 0; s <= todo; ++s) {
            __syncwarp();
            if (s == 0 && automatic) {
                double g = 0.0;
                for (int i = lane; i < n; i += 32)
                    g = fmax(g, (double)re_of(As[i * LD + i]) * (double)re_of(Xs[i * LD + i]));
                for (int d = 16; d > 0; d >>= 1) g = fmax(g, __shfl_xor_sync(0xffffffffu, g, d));
                todo = g > kAutoRefineGamma ? 1 : 0;
            }
            if (s == todo) break;
            // E = I - A X (rows of A from its conjugate: A Hermitian)
            ResidTile<V, TR, TC> et;
            et.init(r0, c0);
#pragma unroll 2
            for (int k = 0; k < TB; ++k) {
                V a[TR], bb[TC];
#pragma unroll
                for (int r = 0; r < TR; ++r) a[r] = conj_v(As[k * LD + r0 + r]);
#pragma unroll
                for (int c = 0; c < TC; ++c) bb[c] = Xs[k * LD + c0 + c];
                et.step(a, bb);
            }
#pragma unroll
            for (int r = 0; r < TR; ++r)
#pragma unroll
                for (int c = 0; c < TC; ++c) Es[(r0 + r) * LD + c0 + c] = et.value(r, c);
            __syncwarp();
            // X + X E, upper half written back
            // (X's rows from its conjugate columns: X Hermitian)
            V acc[TR][TC];
#pragma unroll
            for (int r = 0; r < TR; ++r)
#pragma unroll
                for (int c = 0; c < TC; ++c) acc[r][c] = Xs[(r0 + r) * LD + c0 + c];
            tile_product<V, true, TB>(Xs, Es, r0, c0, acc);
            __syncwarp();  // every lane has read X: its square now takes the new X (mirrored upper half)
#pragma unroll
            for (int r = 0; r < TR; ++r)
#pragma unroll
                for (int c = 0; c < TC; ++c) {
                    const int i = r0 + r, j = c0 + c;
                    if (i <= j && j < n) {
                        const V x = (i == j) ? from_real<V>(re_of(acc[r][c])) : acc[r][c];
                        X[o + gidx(i, j)] = x;
                        Xs[i * LD + j] = x;
                        Xs[j * LD + i] = conj_v(x);
                    }
                }
        }
    }
}

template <typename V, int TB>
static cudaError_t launch_refine_tiled(const BatchParams& p, int steps, int automatic, cudaStream_t s, bool dry) {
    static std::once_flag once;
    static cudaError_t setup = cudaSuccess;
    constexpr int warps = (sizeof(V) == 4 || TB == 16) ? 4 : 2;
    const size_t smem = refine_tiled_warp_bytes<V, TB>() * warps;
    auto kern = k_refine_tiled<V, TB>;
    std::call_once(once, [&] {
        setup = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
    if (setup != cudaSuccess || dry) return setup;
    int per_sm = 1;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * warps, smem);
    if (e != cudaSuccess) return e;
    const int grid = std::max(1, std::min((p.batch + warps - 1) / warps, device_info().sms * std::max(per_sm, 1)));
    kern<<<grid, 32 * warps, smem, s>>>(p, steps, automatic);
    return cudaGetLastError();
}

template <typename V, bool R64>
static cudaError_t launch_refine_r(const BatchParams& p, int steps, int automatic, cudaStream_t s, bool dry) {
    auto kern = k_refine<V, R64>;
    static std::once_flag once;
    static cudaError_t setup = cudaSuccess;
    std::call_once(once, [&] {
        setup = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    });
    if (setup != cudaSuccess || dry) return setup;
    const size_t per = refine_warp_bytes<V>(p.max_n);
    const int warps = (int)std::max<size_t>(1, std::min<size_t>(4, 98304 / per));
    int per_sm = 1;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * warps, per * warps);
    if (e != cudaSuccess) return e;
    const int grid = std::max(1, std::min((p.batch + warps - 1) / warps, device_info().sms * std::max(per_sm, 1)));
    kern<<<grid, 32 * warps, per * warps, s>>>(p, steps, automatic);
    return cudaGetLastError();
}

template <typename V>
static cudaError_t launch_refine_t(const BatchParams& p, int steps, int automatic, cudaStream_t s, bool dry) {
    if (p.flags & CHOL_FLAG_RESIDUAL_FP64) return launch_refine_r<V, true>(p, steps, automatic, s, dry);
    if (p.max_n <= 16) return launch_refine_tiled<V, 16>(p, steps, automatic, s, dry);
    if (p.max_n <= 32) return launch_refine_tiled<V, 32>(p, steps, automatic, s, dry);
    return launch_refine_r<V, false>(p, steps, automatic, s, dry);
}

// The FP64-pivot pass of CHOL_FLAG_PIVOT64_AUTO over the whole batch (k_redo
// in batched.cuh): one warp per matrix, most of which exit at once.
template <typename V>
static cudaError_t launch_redo_t(const BatchParams& p, cudaStream_t s, bool dry) {
    static std::once_flag once;
    static cudaError_t setup = cudaSuccess;
    std::call_once(once, [&] {
        setup = cudaFuncSetAttribute(k_redo<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    });
    if (setup != cudaSuccess || dry) return setup;
    const int smax = p.max_n;
    const size_t per = warp_elems(p, smax) * sizeof(V);
    const int warps = (int)std::max<size_t>(1, std::min<size_t>(8, 98304 / per));
    const int grid = std::max(1, std::min((p.batch + warps - 1) / warps, device_info().sms * 4));
    k_redo<V><<<grid, 32 * warps, per * warps, s>>>(p, smax, warps);
    return cudaGetLastError();
}

template <typename V>
static cudaError_t launch_single_t(const BatchParams& p, int* work, cudaStream_t s, bool dry) {
    static std::once_flag once;
    static cudaError_t setup = cudaSuccess;
    std::call_once(once, [&] {
        setup = cudaFuncSetAttribute(k_warp_all<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    });
    if (setup != cudaSuccess || dry) return setup;
    const int smax = p.max_n;
    const size_t per = warp_elems(p, smax) * sizeof(V);
    const int warps = (int)std::max<size_t>(1, std::min<size_t>(4, 98304 / per));
    int per_sm = 1;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_warp_all<V>, 32 * warps, per * warps);
    if (e != cudaSuccess) return e;
    const int grid = std::max(1, std::min((p.batch + warps - 1) / warps, device_info().sms * std::max(per_sm, 1)));
    k_warp_all<V><<<grid, 32 * warps, per * warps, s>>>(p, smax, warps, work);
    return cudaGetLastError();
}

cudaError_t launch_single(int dtype, const BatchParams& p, int* work, cudaStream_t s, bool dry) {
    switch (dtype) {
        case CHOL_F32: return launch_single_t<float>(p, work, s, dry);
        case CHOL_F64: return launch_single_t<double>(p, work, s, dry);
        case CHOL_C64: return launch_single_t<cpx<float>>(p, work, s, dry);
        case CHOL_C128: return launch_single_t<cpx<double>>(p, work, s, dry);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_redo(int dtype, const BatchParams& p, cudaStream_t s, bool dry) {
    if (dtype == CHOL_F32) return launch_redo_t<float>(p, s, dry);
    if (dtype == CHOL_C64) return launch_redo_t<cpx<float>>(p, s, dry);
    return cudaSuccess;  // FP64 value types form Eq. 3 in FP64 already
}

cudaError_t launch_refine(int dtype, const BatchParams& p, int steps, int automatic, cudaStream_t s, bool dry) {
    if (dtype == CHOL_F32) return launch_refine_t<float>(p, steps, automatic, s, dry);
    if (dtype == CHOL_C64) return launch_refine_t<cpx<float>>(p, steps, automatic, s, dry);
    return cudaErrorInvalidValue;
}

}  // namespace cholinv
