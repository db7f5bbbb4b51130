// Wide kernel: one warp per matrix for FP32 orders 33..64, the matrix in the
// warp's registers.
//
// Lane h owns columns j = h and j = 32 + h and keeps each in full, rows
// 0..N-1 (2N registers): the upper part holds A, then R, then X in place;
// the lower part (rows k > j) receives x_jk once row j of X is known, so
// that every x~_kj of the inverse (x_kj for k <= j, x_jk for k > j) is in
// the owner's registers.  The packed upper triangle in shared memory (the
// "mirror", as in the group kernel) carries each finished row of R or X to
// the other lanes, read with 16-byte broadcast loads.
//   factor (Eqs. 3-4), right-looking: at step k the pivot t_k arrives by a
//     shuffle from column k's owner; row k of R is scaled by the owners of
//     columns j >= k and published; every lane then subtracts
//     r_ki r_kj from rows i > k of its columns, so entry (i, j) receives its
//     terms in ascending k, the order of Eq. 4's sum;
//   inverse (Sec. IV.A), rows N..1: x_ij = -(1/r_ii) sum_{k>i} r_ik x~_kj is
//     a dot product of row i of R (broadcast) with the lane's own column;
//     x_ii = (1/r_ii)(1/r_ii - sum_j r_ij x_ij) takes one warp reduction.
// Rows are template recursions over std::integral_constant, so every
// register index is a compile-time constant (with #pragma unroll alone the
// compiler stops unrolling loops this large and leaves the columns in local
// memory).  Lanes compute every row of both slots without ownership
// predicates: a value a lane computes for a row it does not own lands in
// the lower part of its column, which is rewritten before it is read.
#pragma once

#include <utility>

#include "group.cuh"

namespace cholinv {

constexpr int kWideLo = 33;
constexpr int kWideHi = 64;

template <class F, int... K>
CHOL_D void static_for_seq(F& f, std::integer_sequence<int, K...>) {
    (f(std::integral_constant<int, K>{}), ...);
}
// f(std::integral_constant<int, K>{}) for K = 0, 1, ..., COUNT-1
template <int COUNT, class F>
CHOL_D void static_for(F&& f) {
    static_for_seq(f, std::make_integer_sequence<int, COUNT>{});
}

// f(k, m_rk) for k = FIRST..N-1: row ROW of the packed mirror M, read in
// aligned 16-byte units (the first and last unit may straddle the row's
// ends; those elements are not passed on).  ROW and FIRST are compile-time,
// so the unrolled loops leave only constant indices.
template <int N, int ROW, int FIRST, class F>
CHOL_D void row_for(const float* M, F&& f) {
    constexpr int base = row_base(N, ROW);
    constexpr int e0 = base + FIRST, e1 = base + N;
    constexpr int u0 = e0 / 4, u1 = (e1 + 3) / 4;
#pragma unroll
    for (int u = u0; u < u1; ++u) {
        const float4 w = reinterpret_cast<const float4*>(M)[u];
        const float v[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int z = 0; z < 4; ++z) {
            const int e = u * 4 + z;
            if (e >= e0 && e < e1) f(e - base, v[z]);
        }
    }
}

// 4 warps (4 matrices) per CTA; the mirror layout is the group kernel's with
// G = 32.
template <int N>
using WideCfg = GroupCfg<float, N, 32, 4>;

// Resident CTAs per SM requested from the register allocator: two (255
// registers a thread) where the columns take 2N > 96 registers, three below.
template <int N>
constexpr int wide_minb() { return N <= 48 ? 3 : 2; }

// GATE: CHOL_FLAG_PIVOT64_AUTO's cancellation test.
template <int N, int MINB = wide_minb<N>(), bool GATE = false>
__global__ void __launch_bounds__(128, MINB) k_wide(BatchParams p) {
    static_assert(N >= kWideLo && N <= kWideHi, "the wide kernel covers orders 33..64");
    using C = WideCfg<N>;
    constexpr int TN = C::TN;
    constexpr int THREADS = C::THREADS;
    constexpr int MPC = C::MPC;
    constexpr unsigned FULL = 0xffffffffu;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* mirs = smem_raw;                                                    // [MPC][STRIDE]
    int64_t* s_off = reinterpret_cast<int64_t*>(smem_raw + (size_t)MPC * C::STRIDE);  // [MPC]
    int* s_info = reinterpret_cast<int*>(s_off + MPC);                                 // [MPC]
    float* s_dinv = reinterpret_cast<float*>(s_info + MPC);                            // [MPC][N]
    uint8_t* s_i = reinterpret_cast<uint8_t*>(s_dinv + MPC * N);                       // [TN]
    uint8_t* s_j = s_i + TN;
    uint64_t* s_bar = reinterpret_cast<uint64_t*>(smem_raw + C::BAR_OFF);  // bulk copies of the vectorised path

    const int t = threadIdx.x;
    const int h = t & 31;
    const int q = t >> 5;
    // the phase of s_bar to wait for lives beside it (kept out of registers)
    uint32_t* s_phase = reinterpret_cast<uint32_t*>(s_bar + 1);
    if (t == 0) {
        mbar_init1(s_bar);
        *s_phase = 0;
    }
    for (int e = t; e < TN; e += THREADS) {
        int i = 0;
        while (pidx(N, i + 1, i + 1) <= e && i + 1 < N) ++i;
        s_i[e] = (uint8_t)i;
        s_j[e] = (uint8_t)(e - pidx(N, i, i) + i);
    }
    const int count = class_count(p, N);
    const int nchunks = (count + MPC - 1) / MPC;
    const float* A = static_cast<const float*>(p.A);
    float* Xo = static_cast<float*>(p.X);
    float* Ro = static_cast<float*>(p.R);
    const bool store_R = p.R != nullptr && p.want_inv;
    constexpr bool gate = GATE;
    __syncthreads();

    for (int chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
        const int m = min(MPC, count - chunk * MPC);
        int ok = 1;
        if (t < m) {
            const int64_t b = member_index(p, N, chunk * MPC + t);
            const int64_t o = matrix_offset(p, N, b);
            s_off[t] = o;
            ok = (o % C::U) == 0;
        }
        const bool vec = (__syncthreads_and(ok) != 0) && p.layout == 1 && p.aligned16;
        group_stage<float, N, C>(p, A, mirs, s_off, s_i, s_j, m, vec, s_bar);
        cp_async_wait<0>();
        bool late = false;
        const bool bulk_in = vec && C::TN / C::U > 0;
        if (bulk_in) late = !mbar_wait_bounded(s_bar, *s_phase);
        if (__syncthreads_or(late)) {
            // a bulk copy did not arrive within the bound: report, wait once
            // more (bounded) for the copies in flight, and stop
            if (t == 0) report_error(p.err, CHOL_ERR_TIMEOUT);
            mbar_wait_bounded(s_bar, *s_phase);
            return;
        }
        if (bulk_in && t == 0) *s_phase ^= 1u;  // read again only after later barriers

        const bool live = q < m;
        float* M = reinterpret_cast<float*>(mirs + (size_t)(live ? q : 0) * C::STRIDE);
        float* dinv = s_dinv + q * N;
        // own columns' upper parts (rows r <= j) from the mirror; other rows
        // are don't-care until the inverse fills them
        float col[2][N];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int jj = min(c * 32 + h, N - 1);
#pragma unroll
            for (int r = 0; r < N; ++r)
                if (r <= c * 32 + 31) col[c][r] = M[row_base(N, r) + jj];
        }
        int info = 0;
        bool redo = false;
        // ---------------- factor, Eqs. 3-4 (right-looking, terms in ascending k)
        static_for<N>([&](auto kc) {
            constexpr int K = decltype(kc)::value;
            constexpr int CO = K / 32, HO = K % 32;
            float aKK = 1.f;
            if constexpr (gate) aKK = M[row_base(N, K) + K];  // read before row K is published
            const float tt = __shfl_sync(FULL, col[CO][K], HO);    // Eq. 3 argument after K updates
            if (gate && pivot_cancels(tt, aKK)) redo = true;
            if (info == 0 && !pivot_ok(tt)) info = K + 1;
            float rii, inv;
            pivot_root(tt, rii, inv);
            if (h == 0) dinv[K] = inv;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                if (K <= c * 32 + 31) {
                    const int j = c * 32 + h;
                    const float r = (j == K) ? rii : col[c][K] * inv;  // Eq. 4's division
                    col[c][K] = r;
                    if (live && j >= K && j < N) M[row_base(N, K) + j] = r;
                }
            }
            __syncwarp();
            if constexpr (K + 1 < N) {
                row_for<N, K, K + 1>(M, [&](int I, float rKi) {
#pragma unroll
                    for (int c = 0; c < 2; ++c)
                        if (I <= c * 32 + 31) col[c][I] = fmaf(-rKi, col[c][K], col[c][I]);
                });
            }
        });
        if (live && h == 0) s_info[q] = redo ? kInfoRedo : info;
        if (store_R || !p.want_inv) {
            __syncthreads();
            group_store<float, N, C, GATE>(p, Ro, mirs, s_off, s_info, s_i, s_j, m, vec, true, false, true);
            __syncthreads();
        }
        if (p.want_inv) {
            // ---------------- proposed inverse, Sec. IV.A, rows N..1
            static_for<N>([&](auto ic) {
                constexpr int I = N - 1 - decltype(ic)::value;
                constexpr int CO = I / 32, HO = I % 32;
                const float inv = dinv[I];
                // two partial sums per column (even and odd k) for independent FMA chains
                float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
                if constexpr (I + 1 < N) {
                    row_for<N, I, I + 1>(M, [&](int K, float rIk) {
#pragma unroll
                        for (int c = 0; c < 2; ++c)
                            if (c * 32 + 31 > I) acc[c][K & 1] = fmaf(rIk, col[c][K], acc[c][K & 1]);
                    });
                }
                float sd = 0.f;
                float xs[2] = {0.f, 0.f};
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    if (c * 32 + 31 > I) {
                        const int j = c * 32 + h;
                        xs[c] = -(acc[c][0] + acc[c][1]) * inv;
                        if (j > I && j < N) sd = fmaf(col[c][I], xs[c], sd);  // r_ij x_ij
                    }
                }
                __syncwarp();  // row I of R has been read by every lane
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    if (c * 32 + 31 > I) {
                        const int j = c * 32 + h;
                        col[c][I] = xs[c];
                        if (live && j > I && j < N) M[row_base(N, I) + j] = xs[c];
                    }
                }
#pragma unroll
                for (int d = 16; d > 0; d >>= 1) sd += __shfl_xor_sync(FULL, sd, d);
                const float xd = (inv - sd) * inv;
                if (h == HO) {
                    col[CO][I] = xd;
                    if (live) M[row_base(N, I) + I] = xd;
                }
                __syncwarp();
                if constexpr (I > 0 && I + 1 < N) {
                    // row I of X into the lower part of column I, on its owner
                    row_for<N, I, I + 1>(M, [&](int K, float x) {
                        if (h == HO) col[CO][K] = x;
                    });
                }
            });
            __syncthreads();
            group_store<float, N, C, GATE>(p, Xo, mirs, s_off, s_info, s_i, s_j, m, vec, false, p.fill_lower != 0,
                                        true);
        }
        if (p.info)
            for (int k = t; k < m; k += THREADS) p.info[member_index(p, N, chunk * MPC + k)] = s_info[k];
        fence_async_smem();  // the next chunk's bulk copies overwrite the mirrors
        __syncthreads();
    }
}

}  // namespace cholinv

// ---------------------------------------------------------------------------
// Host side: launch the order-N kernel over class N's members (persistent
// grid: at most the resident CTAs of every SM).
// ---------------------------------------------------------------------------
#include <algorithm>
#include <mutex>

#include "dispatch.h"

namespace cholinv {

template <int N, bool GATE>
static cudaError_t launch_wide_t(const BatchParams& p, int upper_count, cudaStream_t s, bool dry) {
    using C = WideCfg<N>;
    auto kern = k_wide<N, wide_minb<N>(), GATE>;
    static std::once_flag once;
    static int per_sm = 1;
    static cudaError_t setup_err = cudaSuccess;
    std::call_once(once, [&] {
        setup_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        if (setup_err == cudaSuccess)
            setup_err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, C::THREADS, C::SMEM);
        if (per_sm < 1) per_sm = 1;
    });
    if (setup_err != cudaSuccess || dry) return setup_err;
    const int chunks = (upper_count + C::MPC - 1) / C::MPC;
    if (chunks <= 0) return cudaSuccess;
    const int grid = std::min(chunks, device_info().sms * per_sm);
    kern<<<grid, C::THREADS, C::SMEM, s>>>(p);
    return cudaGetLastError();
}

template <int N>
static cudaError_t launch_wide(const BatchParams& p, int upper_count, cudaStream_t s, bool dry) {
    if (p.flags & CHOL_FLAG_PIVOT64_AUTO) return launch_wide_t<N, true>(p, upper_count, s, dry);
    return launch_wide_t<N, false>(p, upper_count, s, dry);
}

// Class `cls` if it lies in [LO, HI] (compile-time recursion).
template <int LO, int HI>
static cudaError_t launch_wide_range(const BatchParams& p, int cls, int upper_count, cudaStream_t s, bool dry) {
    if constexpr (HI < LO) {
        return cudaErrorInvalidValue;
    } else {
        if (cls == HI) return launch_wide<HI>(p, upper_count, s, dry);
        return launch_wide_range<LO, HI - 1>(p, cls, upper_count, s, dry);
    }
}

}  // namespace cholinv
