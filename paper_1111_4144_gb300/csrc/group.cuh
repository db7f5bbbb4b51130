// Group kernel: G threads (a power of two, G <= 32) share one matrix.
//
// Thread h of a group owns the columns j = c*G + h (c = 0..NC-1) and keeps
// their upper parts in registers: first the columns of A, then of R, then of
// X, each replacing the last in place.  A copy of the packed upper triangle
// in shared memory (the matrix's "mirror") carries what a thread needs from
// columns it does not own:
//   Eq. 4, row i      needs column i of R above the diagonal  -> read from the mirror
//   Sec. IV.A, row i  needs row i of R and, for x~_kj with k > j, row j of X
//                                                            -> read from the mirror
// Every new row of R or X is written to the mirror as it is produced, so at
// the end the mirror holds the result and is stored with coalesced copies.
// Rows are fully unrolled (N compile-time), so every register index is a
// compile-time constant; ownership tests on the runtime lane index become
// predicates, not branches.
#pragma once

#include <type_traits>

#include "batched.cuh"

namespace cholinv {

template <typename V, int N, int G, int W = 4>
struct GroupCfg {
    static_assert(G >= 2 && G <= 32 && (G & (G - 1)) == 0, "G must be a power of two in [2, 32]");
    static_assert(W % 4 == 0, "whole warps per SM sub-partition");
    static constexpr int TN = tri(N);
    static constexpr int NC = (N + G - 1) / G;   // columns per thread
    static constexpr int MPW = 32 / G;           // matrices per warp
    static constexpr int WARPS = W;
    static constexpr int THREADS = 32 * WARPS;
    static constexpr int MPC = MPW * WARPS;       // matrices per CTA chunk
    // bytes of one matrix's mirror, in whole 16-byte units.  A warp access is
    // served 128 bytes at a time, and its groups touch the same offsets of
    // consecutive mirrors (a broadcast per group) or G consecutive elements
    // each; a mirror stride of +-G elements modulo 128 bytes lays the groups
    // of one 128-byte phase side by side over all banks, for both patterns
    // and for the rows of X read in the inverse.  When G elements are not a
    // multiple of 16 bytes (or fill 128), an odd number of units.
    static constexpr int UNITS0 = (TN * (int)sizeof(V) + 15) / 16;
    static constexpr int stride_units() {
        constexpr int gb = (G * (int)sizeof(V)) % 128;
        int u = UNITS0;
        const bool odd = gb == 0 || gb % 16 != 0;
        while (!odd && (u * 16) % 128 != gb && (u * 16) % 128 != 128 - gb) ++u;
        return odd ? (u % 2 ? u : u + 1) : u;
    }
    static constexpr int UNITS = stride_units();
    static constexpr int STRIDE = UNITS * 16;
    static constexpr int U = 16 / (int)sizeof(V);
    // 32-bit words of the owned columns' upper parts (rows 0..c*G+G-1 of slot c)
    static constexpr int colw() {
        int w = 0;
        for (int c = 0; c < NC; ++c) w += (c * G + G < N ? c * G + G : N);
        return w * (int)(sizeof(V) / 4);
    }
    static constexpr int COLW = colw();
    // the mbarrier of the bulk copies (8-byte aligned) after the other arrays
    static constexpr size_t BAR_OFF = ((size_t)MPC * STRIDE + (size_t)MPC * (sizeof(int64_t) + sizeof(int)) +
                                       (size_t)MPC * N * sizeof(typename traits<V>::real) + 2 * (size_t)TN + 7) / 8 * 8;
    static constexpr size_t SMEM = BAR_OFF + 16;  // the mbarrier and its phase
};

// ---------------------------------------------------------------------------
// Bulk asynchronous copies (the untiled TMA form) of whole packed matrices
// between global memory and the mirrors: one copy per matrix instead of one
// cp.async per 16-byte unit.  Loads complete on an mbarrier whose wait is
// bounded (about one second of %globaltimer); both ends of every copy are
// 16-byte aligned and its size a multiple of 16 (the vectorised path only).
// ---------------------------------------------------------------------------
CHOL_D void mbar_init1(uint64_t* b) {
    asm volatile("mbarrier.init.shared.b64 [%0], 1;" ::"r"(smem_u32(b)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
CHOL_D void mbar_arrive_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes)
                 : "memory");
}
CHOL_D bool mbar_done(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
CHOL_D uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
// true once the phase with this parity has completed; false after ~1 s
CHOL_D bool mbar_wait_bounded(uint64_t* b, uint32_t parity) {
    const uint64_t t0 = global_ns();
    while (!mbar_done(b, parity))
        if (global_ns() - t0 > 1000000000ull) return false;
    return true;
}
CHOL_D void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
CHOL_D void bulk_s2g(void* dst, const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// the shared-memory source of this thread's bulk stores may be reused
CHOL_D void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// order this thread's generic shared-memory accesses before later async-proxy ones
CHOL_D void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Copy the chunk's matrices into the mirrors (cp.async, not waited on).
// C supplies THREADS, TN, U (elements per 16-byte unit) and STRIDE.
// bar (optional): the vectorised path copies each matrix's whole units with
// one bulk copy completing on *bar (the caller waits on it); the remaining
// elements, and every element without bar, by cp.async.
template <typename V, int N, class C>
CHOL_D void group_stage(const BatchParams& p, const V* A, unsigned char* mir, const int64_t* s_off,
                        const uint8_t* s_i, const uint8_t* s_j, int m, bool vec, uint64_t* bar = nullptr) {
    const int t = threadIdx.x;
    if (vec) {
        constexpr int FULL = C::TN / C::U;  // whole units per matrix
        constexpr int TAIL = C::TN - FULL * C::U;
        if (bar != nullptr && FULL > 0) {
            if (t == 0) mbar_arrive_tx(bar, (uint32_t)m * FULL * 16);
            if (t < m) bulk_g2s(mir + (size_t)t * C::STRIDE, A + s_off[t], FULL * 16, bar);
        } else {
            for (int f = t; f < m * FULL; f += C::THREADS) {
                const int q = f / FULL, u = f - q * FULL;
                cp_async<16>(mir + (size_t)q * C::STRIDE + u * 16, A + s_off[q] + u * C::U);
            }
        }
        if constexpr (TAIL > 0) {
            for (int f = t; f < m * TAIL; f += C::THREADS) {
                const int q = f / TAIL, r = f - q * TAIL;
                const int e = FULL * C::U + r;
                cp_async<(int)sizeof(V)>(mir + (size_t)q * C::STRIDE + e * sizeof(V), A + s_off[q] + e);
            }
        }
    } else {
        for (int f = t; f < m * C::TN; f += C::THREADS) {
            const int q = f / C::TN, e = f - q * C::TN;
            const int64_t g = p.layout ? (int64_t)e : (int64_t)s_i[e] * N + s_j[e];
            cp_async<(int)sizeof(V)>(mir + (size_t)q * C::STRIDE + e * sizeof(V), A + s_off[q] + g);
        }
    }
    cp_async_commit();
}

// Store the mirrors (X, or R when factoring) to global memory.  GATE:
// matrices marked kInfoRedo are skipped (CHOL_FLAG_PIVOT64_AUTO).
// bulk (optional): the vectorised path stores each matrix's whole units
// with one bulk copy (a failed matrix's mirror is first filled with NaN);
// the caller has synchronised the CTA after the mirror's last write.
template <typename V, int N, class C, bool GATE = false>
CHOL_D void group_store(const BatchParams& p, V* out, unsigned char* mir, const int64_t* s_off,
                        const int* s_info, const uint8_t* s_i, const uint8_t* s_j, int m, bool vec, bool is_factor,
                        bool fill_lower, bool bulk = false) {
    const int t = threadIdx.x;
    if (vec) {
        constexpr int FULL = C::TN / C::U;
        constexpr int TAIL = C::TN - FULL * C::U;
        if (bulk && FULL > 0) {
            const bool skip = t >= m || (GATE && s_info[t] == kInfoRedo);
            if (!skip && s_info[t] != 0) {
                uint4 qn;
#pragma unroll
                for (int r = 0; r < C::U; ++r) reinterpret_cast<V*>(&qn)[r] = nan_v<V>();
                for (int u = 0; u < FULL; ++u) *reinterpret_cast<uint4*>(mir + (size_t)t * C::STRIDE + u * 16) = qn;
            }
            fence_async_smem();
            __syncthreads();
            if (!skip) {
                bulk_s2g(out + s_off[t], mir + (size_t)t * C::STRIDE, FULL * 16);
                bulk_wait_read();
            }
        }
        for (int f = t; f < ((bulk && FULL > 0) ? 0 : m * FULL); f += C::THREADS) {
            const int q = f / FULL, u = f - q * FULL;
            if constexpr (GATE)
                if (s_info[q] == kInfoRedo) continue;  // left to the FP64-pivot pass
            uint4 v = *reinterpret_cast<const uint4*>(mir + (size_t)q * C::STRIDE + u * 16);
            if (s_info[q] != 0) {
                const V qn = nan_v<V>();
#pragma unroll
                for (int r = 0; r < C::U; ++r) reinterpret_cast<V*>(&v)[r] = qn;
            }
            *reinterpret_cast<uint4*>(out + s_off[q] + u * C::U) = v;
        }
        if constexpr (TAIL > 0) {
            for (int f = t; f < m * TAIL; f += C::THREADS) {
                const int q = f / TAIL, r = f - q * TAIL;
                if constexpr (GATE)
                    if (s_info[q] == kInfoRedo) continue;
                const int e = FULL * C::U + r;
                const V v = *reinterpret_cast<const V*>(mir + (size_t)q * C::STRIDE + e * sizeof(V));
                out[s_off[q] + e] = s_info[q] ? nan_v<V>() : v;
            }
        }
    } else {
        for (int f = t; f < m * C::TN; f += C::THREADS) {
            const int q = f / C::TN, e = f - q * C::TN;
            if constexpr (GATE)
                if (s_info[q] == kInfoRedo) continue;
            const int64_t o = s_off[q];
            const int i = s_i[e], j = s_j[e];
            const bool bad = s_info[q] != 0;
            const V v = bad ? nan_v<V>() : *reinterpret_cast<const V*>(mir + (size_t)q * C::STRIDE + e * sizeof(V));
            if (p.layout) {
                out[o + e] = v;
            } else {
                out[o + (int64_t)i * N + j] = v;
                if (i != j) {
                    if (is_factor) out[o + (int64_t)j * N + i] = bad ? nan_v<V>() : zero_v<V>();
                    else if (fill_lower) out[o + (int64_t)j * N + i] = conj_v(v);
                }
            }
        }
    }
}

// Offset (in elements) of row r of the packed upper mirror, minus r, so that
// element (r, j) sits at row_base(r) + j.
CHOL_HD constexpr int row_base(int n, int r) { return r * n - (r * (r - 1)) / 2 - r; }

// Row r of the packed mirror, columns r..N-1, into out[r..N-1], using 16-byte
// loads wherever a whole aligned unit lies inside the row.
template <typename V, int N>
CHOL_D void load_row(const V* M, int r, V (&out)[N]) {
    constexpr int U = 16 / (int)sizeof(V);
#pragma unroll
    for (int k = 0; k < N; ++k) {
        if (k >= r) {
            const int e = row_base(N, r) + k;
            // a unit may run past the row's end into the next row (or the
            // mirror's padding); those extra elements are not used
            const bool unit_start = (e % U) == 0;
            const bool in_unit = (e % U) != 0 && k - (e % U) >= r;  // covered by an earlier unit load
            if (unit_start) {
                const uint4 w = *reinterpret_cast<const uint4*>(M + e);
#pragma unroll
                for (int z = 0; z < U; ++z)
                    if (k + z < N) out[k + z] = reinterpret_cast<const V*>(&w)[z];
            } else if (!in_unit) {
                out[k] = M[e];
            }
        }
    }
}

// Per-row synchronisation of a group: a warp barrier, or (ALG 3) a CTA
// barrier that also keeps the CTA's warps on the same stretch of code.
template <int ALG>
CHOL_D void row_sync() {
    if constexpr (ALG == 3) __syncthreads(); else __syncwarp();
}

// Threads per matrix for order N (ALG 1): the smallest power of two
// (2..32) whose share of the columns' upper parts fits in about 150 32-bit
// registers; 0 if none does (the one-matrix-per-warp kernel takes those).
// Fewer threads per matrix measured faster (less repeated mirror traffic)
// even at lower occupancy: for 16 x 16 complex64, G = 2 / 4 / 8 / 16 took
// 276 / 345 / 493 / 700 us per 349,525 matrices on one GB300.
template <typename V, int N>
constexpr int group_size() {
    for (int g = 2; g <= 32; g *= 2) {
        int words = 0;
        const int nc = (N + g - 1) / g;
        for (int c = 0; c < nc; ++c) words += (c * g + g < N ? c * g + g : N) * traits<V>::words;
        if (words <= 150) return g;
    }
    return 0;
}

// ALG 1: left-looking Eq. 4 (column i of R read from the mirror at row i);
//        inverse terms with k > j read row j of X from the mirror.  For
//        complex64 the sums run on paired FP32 instructions (below) when the
//        owned columns plus the paired accumulators fit the register budget:
//        in the factor, and in the inverse too without a register cap
//        (MINB = 1).
//        On one GB300 (349,525 matrices) this took order 16 from 313 to
//        306 us (factor only; the inverse's accumulators spill under the
//        128-register cap) and order 8 from 56.4-57.2 to 55.4 us.
// ALG 2 (an alternative kept for tuning; it ignores CHOL_FLAG_PIVOT64 and
//        is not dispatched by default): the same sums taken right-looking (row k of R broadcast from the
//        mirror, each entry still receives its terms in ascending k); in the
//        inverse every thread keeps its columns in full (the lower half
//        mirrored in once per row), so the dot products run on registers.
// GATE: CHOL_FLAG_PIVOT64_AUTO's cancellation test (FP32 value types only).
template <typename V, int N, int G, int ALG, int W = 4, int MINB = 1, bool GATE = false, bool LDL = false,
          bool P64 = false>
__global__ void __launch_bounds__(GroupCfg<V, N, G, W>::THREADS, MINB)
k_group(BatchParams p) {
    static_assert(!LDL || ALG == 1, "the LDL form is built on the left-looking rows");
    using C = GroupCfg<V, N, G, W>;
    using R = typename traits<V>::real;
    constexpr int NC = C::NC;
    constexpr int TN = C::TN;
    constexpr int THREADS = C::THREADS;
    constexpr int MPC = C::MPC;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* mirs = smem_raw;                                              // [MPC][STRIDE]
    int64_t* s_off = reinterpret_cast<int64_t*>(smem_raw + (size_t)MPC * C::STRIDE);  // [MPC]
    int* s_info = reinterpret_cast<int*>(s_off + MPC);                           // [MPC]
    R* s_dinv = reinterpret_cast<R*>(s_info + MPC);                              // [MPC][N] (MINB > 1)
    uint8_t* s_i = reinterpret_cast<uint8_t*>(s_dinv + MPC * N);                 // [TN]
    uint8_t* s_j = s_i + TN;
    uint64_t* s_bar = reinterpret_cast<uint64_t*>(smem_raw + C::BAR_OFF);  // bulk copies of the vectorised path

    const int t = threadIdx.x;
    const int lane = t & 31;
    const int h = t & (G - 1);           // position in the group
    const int q = t / G;                 // matrix within the chunk
    const int gbase = lane & ~(G - 1);   // first lane of this group
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
    const V* A = static_cast<const V*>(p.A);
    V* Xo = static_cast<V*>(p.X);
    V* Ro = static_cast<V*>(p.R);
    const bool store_R = p.R != nullptr && p.want_inv;
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
        group_stage<V, N, C>(p, A, mirs, s_off, s_i, s_j, m, vec, s_bar);
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

        if constexpr (ALG == 1 || ALG == 3) {
        // A complex product a b splits over the parts of a:
        //   a b = {a.re, a.re} o {b.re, b.im} + {a.im, a.im} o {-b.im, b.re},
        // so a sum of products is carried as P = sum {a.re, a.re} o b and
        // Q = sum {a.im, a.im} o b (one paired FMA each per term, two
        // independent chains) and combined once per entry.
        constexpr bool kC64 = std::is_same<V, cpx<float>>::value;
        // the paired accumulators (4 words per owned column) on top of the
        // columns must leave the columns in registers; measured to help with
        // G <= 4 only
        constexpr bool kPair = kC64 && G <= 4 && C::COLW + 4 * NC <= 96;    // factor
        constexpr bool kPairI = kPair && MINB == 1;                         // inverse
        const bool live = q < m;
        V* M = reinterpret_cast<V*>(mirs + (size_t)(live ? q : 0) * C::STRIDE);
        // own columns, upper parts, into registers
        V col[NC][N];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int j = c * G + h;
            const int jj = min(j, N - 1);
#pragma unroll
            for (int r = 0; r < N; ++r) {
                if (r <= c * G + G - 1) {
                    const V v = M[row_base(N, r) + jj];
                    col[c][r] = (r <= j && j < N) ? v : zero_v<V>();
                }
            }
        }
        // 1/r_ii of every row: in registers, or (register-capped variants) in
        // shared memory, written by the owner of row i and read by the group
        constexpr bool kDinvShared = MINB > 1;
        R dinv_r[kDinvShared ? 1 : N];
        R* dinv_s = s_dinv + (live ? q : 0) * N;
        auto dinv_put = [&](int i, R v) {
            if constexpr (kDinvShared) {
                if (live && h == i % G) dinv_s[i] = v;
            } else {
                dinv_r[i] = v;
            }
        };
        auto dinv_get = [&](int i) -> R {
            if constexpr (kDinvShared) return dinv_s[i]; else return dinv_r[i];
        };
        int info = 0;
        bool redo = false;
        constexpr bool gate = GATE;
        // LDL (Sec. II.A, Eqs. 9-11): d_k of the rows done, and R unit upper
        // with d_i on its diagonal; the mirror's column i is scaled by d_k
        // before it enters the sums of Eq. 11, whose j = i term is Eq. 10's d_i
        R dd[LDL ? N : 1];
        // ---------------- factor, Eqs. 3-4, row by row
#pragma unroll
        for (int i = 0; i < N; ++i) {
            // a_ii, for the cancellation test (row i of the mirror is written at the end of this step)
            R aii = R(1);
            if constexpr (gate) aii = re_of(M[row_base(N, i) + i]);
            V ci[kPair ? 1 : N];  // column i above the diagonal, from the mirror
            V sv[NC];
            if constexpr (kPair) {
                // s - sum_k conj(r_ki) r_kj: P starts at s and takes -r_ki.re,
                // Q takes r_ki.im; then s = {P.x - Q.y, P.y + Q.x}
                float2 P[NC], Q[NC];
#pragma unroll
                for (int c = 0; c < NC; ++c)
                    if (i <= c * G + G - 1) P[c] = make_float2(re_of(col[c][i]), col[c][i].im);
#pragma unroll
                for (int k = 0; k < N; ++k) {
                    if (k < i) {
                        V a = M[row_base(N, k) + i];
                        if constexpr (LDL) a = scale_v(a, dd[k]);
                        const float2 nar = make_float2(-a.re, -a.re), aim = make_float2(a.im, a.im);
#pragma unroll
                        for (int c = 0; c < NC; ++c) {
                            if (i <= c * G + G - 1) {
                                const float2 b = make_float2(col[c][k].re, col[c][k].im);
                                P[c] = __ffma2_rn(nar, b, P[c]);
                                Q[c] = k == 0 ? __fmul2_rn(aim, b) : __ffma2_rn(aim, b, Q[c]);
                            }
                        }
                    }
                }
#pragma unroll
                for (int c = 0; c < NC; ++c)
                    if (i <= c * G + G - 1)
                        sv[c] = i == 0 ? col[c][i] : V{P[c].x - Q[c].y, P[c].y + Q[c].x};
            } else {
#pragma unroll
                for (int k = 0; k < N; ++k) {
                    if (k < i) {
                        ci[k] = M[row_base(N, k) + i];
                        if constexpr (LDL) ci[k] = scale_v(ci[k], dd[k]);
                    }
                }
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    if (i <= c * G + G - 1) {
                        V s = col[c][i];
#pragma unroll
                        for (int k = 0; k < N; ++k)
                            if (k < i) s = fnma_conj(ci[k], col[c][k], s);
                        sv[c] = s;
                    }
                }
            }
            const int co = i / G, ho = i % G;
            const R tc = re_of(sv[co]);
            const R tt = __shfl_sync(0xffffffffu, tc, gbase + ho);
            R rii, inv;
            if constexpr (LDL) {
                if (info == 0 && !pivot_ok(tt)) info = i + 1;
                rii = tt;  // d_i
                inv = R(1) / tt;
                dd[i] = tt;
            } else if constexpr (sizeof(R) == 4 && P64) {
                // Eq. 3 in FP64: a_ii (still in the mirror) minus |r_ki|^2 over column i
                double td = (double)re_of(M[row_base(N, i) + i]);
#pragma unroll
                for (int k = 0; k < N; ++k) {
                    if (k < i) {
                        if constexpr (kPair) td -= pivot64_term(M[row_base(N, k) + i]);
                        else td -= pivot64_term(ci[k]);
                    }
                }
                if (info == 0 && !pivot_ok(td)) info = i + 1;
                pivot_root64(td, rii, inv);
            } else {
                if (gate && pivot_cancels(tt, aii)) redo = true;
                if (info == 0 && !pivot_ok(tt)) info = i + 1;
                pivot_root(tt, rii, inv);
            }
            dinv_put(i, inv);
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                if (i <= c * G + G - 1) {
                    const int j = c * G + h;
                    if (j < N && j >= i) {
                        const V r = (j == i) ? from_real<V>(rii) : scale_v(sv[c], inv);
                        col[c][i] = r;
                        if (live) M[row_base(N, i) + j] = r;
                    }
                }
            }
            row_sync<ALG>();
        }
        if (live && h == 0) s_info[q] = redo ? kInfoRedo : info;
        if (store_R || !p.want_inv) {
            __syncthreads();
            group_store<V, N, C, GATE>(p, Ro, mirs, s_off, s_info, s_i, s_j, m, vec, true, false, true);
            __syncthreads();
        }
        if (p.want_inv) {
            // ---------------- proposed inverse, Sec. IV.A, rows N..1
#pragma unroll
            for (int i = N - 1; i >= 0; --i) {
                V rr[kPairI ? 1 : N];  // row i of R (16-byte loads where a whole unit lies in the row)
                if constexpr (!kPairI) load_row<V, N>(M, i, rr);
                const R inv = dinv_get(i);
                V xs[NC];
                R sd = R(0);
                if constexpr (kPairI) {
                    // sum_{k>i} r_ik x~_kj as P = sum {r.re, r.re} o x~,
                    // Q = sum {r.im, r.im} o x~, sum = {P.x - Q.y, P.y + Q.x};
                    // row i of R read in 16-byte units as k advances
                    float2 P[NC], Q[NC];
                    V carry = zero_v<V>();
#pragma unroll
                    for (int k = 0; k < N; ++k) {
                        if (k > i) {
                            const int e = row_base(N, i) + k;
                            V r;
                            if (e % 2 == 0) {
                                const uint4 w = *reinterpret_cast<const uint4*>(M + e);
                                r = reinterpret_cast<const V*>(&w)[0];
                                carry = reinterpret_cast<const V*>(&w)[1];
                            } else if (k == i + 1) {
                                const uint4 w = *reinterpret_cast<const uint4*>(M + e - 1);
                                r = reinterpret_cast<const V*>(&w)[1];
                            } else {
                                r = carry;
                            }
                            const float2 rre = make_float2(r.re, r.re), rim = make_float2(r.im, r.im);
#pragma unroll
                            for (int c = 0; c < NC; ++c) {
                                if (c * G + G - 1 > i) {
                                    const int j = c * G + h;
                                    const int jb = row_base(N, min(j, N - 1));
                                    V xt;
                                    if (k <= c * G) {
                                        xt = col[c][k];
                                    } else if (k > c * G + G - 1) {
                                        xt = conj_v(M[jb + k]);
                                    } else {
                                        xt = (k <= j) ? col[c][k] : conj_v(M[jb + k]);
                                    }
                                    const float2 b = make_float2(xt.re, xt.im);
                                    P[c] = k == i + 1 ? __fmul2_rn(rre, b) : __ffma2_rn(rre, b, P[c]);
                                    Q[c] = k == i + 1 ? __fmul2_rn(rim, b) : __ffma2_rn(rim, b, Q[c]);
                                }
                            }
                        }
                    }
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        if (c * G + G - 1 > i) {
                            const int j = c * G + h;
                            const V acc = i + 1 < N ? V{P[c].x - Q[c].y, P[c].y + Q[c].x} : zero_v<V>();
                            xs[c] = LDL ? -acc : scale_v(acc, -inv);
                            if (j > i && j < N) sd = fma_re_conjb(col[c][i], xs[c], sd);
                        }
                    }
                } else {
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    if (c * G + G - 1 > i) {
                        const int j = c * G + h;
                        const bool act = j > i && j < N;
                        const int jb = row_base(N, min(j, N - 1));
                        V acc = zero_v<V>();
#pragma unroll
                        for (int k = 0; k < N; ++k) {
                            if (k > i) {
                                V xt;
                                if (k <= c * G) {
                                    xt = col[c][k];                       // k <= j: own column, row k
                                } else if (k > c * G + G - 1) {
                                    xt = conj_v(M[jb + k]);               // k > j: row j of X
                                } else {
                                    xt = (k <= j) ? col[c][k] : conj_v(M[jb + k]);
                                }
                                acc = fma_v(rr[k], xt, acc);
                            }
                        }
                        xs[c] = LDL ? -acc : scale_v(acc, -inv);
                        // diagonal partial: r_ij conj(x_ij) over own columns
                        if (act) sd = fma_re_conjb(col[c][i], xs[c], sd);
                    }
                }
                }
                row_sync<ALG>();  // row i of R is read; it may now be overwritten
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    if (c * G + G - 1 > i) {
                        const int j = c * G + h;
                        if (j > i && j < N) {
                            col[c][i] = xs[c];
                            if (live) M[row_base(N, i) + j] = xs[c];
                        }
                    }
                }
#pragma unroll
                for (int d = G / 2; d > 0; d >>= 1) sd += __shfl_xor_sync(0xffffffffu, sd, d);
                const V xd = from_real<V>(LDL ? inv - sd : (inv - sd) * inv);
                const int co = i / G, ho = i % G;
                if (h == ho) {
                    col[co][i] = xd;
                    if (live) M[row_base(N, i) + i] = xd;
                }
                row_sync<ALG>();
            }
            __syncthreads();
            group_store<V, N, C, GATE>(p, Xo, mirs, s_off, s_info, s_i, s_j, m, vec, false, p.fill_lower != 0,
                                        true);
        }
        } else {
        const bool live = q < m;
        V* M = reinterpret_cast<V*>(mirs + (size_t)(live ? q : 0) * C::STRIDE);
        // Own columns in registers.  col[c][r] holds row r of column j = c*G + h:
        // rows r <= j first hold A, then R, then X (each in place); rows r > j
        // receive the mirrored lower half of X, conj(x_jr), once row j of X is done.
        V col[NC][N];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int j = c * G + h;
            const int jj = min(j, N - 1);
#pragma unroll
            for (int r = 0; r < N; ++r) {
                if (r <= c * G + G - 1) {
                    const V v = M[row_base(N, r) + jj];
                    col[c][r] = (r <= j && j < N) ? v : zero_v<V>();
                }
            }
        }
        int info = 0;
        // ---------------- factor, Eqs. 3-4.  Entry (i, j) receives its terms
        // conj(r_ki) r_kj in the order k = 0, 1, ..., i-1 (one per step k, as
        // in Eq. 4's sum), then the scaling by 1/r_ii at step i.
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const int co = k / G, ho = k % G;
            const R tt = __shfl_sync(0xffffffffu, re_of(col[co][k]), gbase + ho);  // Eq. 3 argument
            if (info == 0 && !pivot_ok(tt)) info = k + 1;
            R rii, inv;
            pivot_root(tt, rii, inv);
            // row k of R in the owned columns (Eq. 4's division), into the mirror
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                if (k <= c * G + G - 1) {
                    const int j = c * G + h;
                    if (j >= k && j < N) {
                        const V r = (j == k) ? from_real<V>(rii) : scale_v(col[c][k], inv);
                        col[c][k] = r;
                        if (live) M[row_base(N, k) + j] = r;
                    }
                }
            }
            __syncwarp();
            if (k + 1 < N) {
                // row k of R (columns > k) for the updates of rows k+1..j
                V rk[N];
                load_row<V, N>(M, k, rk);
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const int j = c * G + h;
#pragma unroll
                    for (int i = 0; i < N; ++i) {
                        if (i > k && i <= c * G + G - 1) {
                            const V u = fnma_conj(rk[i], col[c][k], col[c][i]);
                            if (i <= c * G) col[c][i] = u;          // i <= j for every h
                            else col[c][i] = (i <= j) ? u : col[c][i];
                        }
                    }
                }
            }
        }
        if (live && h == 0) s_info[q] = info;
        if (store_R || !p.want_inv) {
            __syncthreads();
            group_store<V, N, C>(p, Ro, mirs, s_off, s_info, s_i, s_j, m, vec, true, false);
            __syncthreads();
        }
        if (p.want_inv) {
            // ---------------- proposed inverse, Sec. IV.A, rows N..1.  At step i
            // every row k > i of an owned column already holds x~_kj, so
            //   x_ij = -(1/r_ii) sum_{k>i} r_ik col[c][k]
            // is a dot product of row i of R (from the mirror) with registers.
#pragma unroll
            for (int i = N - 1; i >= 0; --i) {
                V rr[N];  // row i of R, columns i..N-1
                load_row<V, N>(M, i, rr);
                const R inv = R(1) / re_of(rr[i]);
                V xs[NC];
                R sd = R(0);
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    if (c * G + G - 1 > i) {
                        const int j = c * G + h;
                        V acc = zero_v<V>();
#pragma unroll
                        for (int k = 0; k < N; ++k)
                            if (k > i) acc = fma_v(rr[k], col[c][k], acc);
                        xs[c] = scale_v(acc, -inv);
                        if (j > i && j < N) sd = fma_re_conjb(col[c][i], xs[c], sd);
                    }
                }
                __syncwarp();  // row i of R has been read; it may be overwritten
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    if (c * G + G - 1 > i) {
                        const int j = c * G + h;
                        if (j > i && j < N) {
                            col[c][i] = xs[c];
                            if (live) M[row_base(N, i) + j] = xs[c];
                        }
                    }
                }
#pragma unroll
                for (int d = G / 2; d > 0; d >>= 1) sd += __shfl_xor_sync(0xffffffffu, sd, d);
                const V xd = from_real<V>((inv - sd) * inv);
                const int co = i / G, ho = i % G;
                if (h == ho) {
                    col[co][i] = xd;
                    if (live) M[row_base(N, i) + i] = xd;
                }
                __syncwarp();
                if (i > 0) {
                    // row i of X is complete: its owner mirrors it into the
                    // lower half of column i (rows k > i hold conj(x_ik))
                    V xr[N];
                    load_row<V, N>(M, i, xr);
#pragma unroll
                    for (int k = 0; k < N; ++k)
                        if (k > i) col[co][k] = (h == ho) ? conj_v(xr[k]) : col[co][k];
                }
            }
            __syncthreads();
            group_store<V, N, C>(p, Xo, mirs, s_off, s_info, s_i, s_j, m, vec, false, p.fill_lower != 0);
        }
        }
        if (p.info)
            for (int k = t; k < m; k += THREADS) p.info[member_index(p, N, chunk * MPC + k)] = s_info[k];
        fence_async_smem();  // the next chunk's bulk copies overwrite the mirrors
        __syncthreads();
    }
}

}  // namespace cholinv
