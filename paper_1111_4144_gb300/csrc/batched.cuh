// Batched factor + direct inverse kernels for small matrices (order <= 64).
//
// Two kernel families, both launched once per size class N:
//   lane kernels (one matrix per thread, N compile-time, fully unrolled):
//     a CTA stages THREADS matrices into shared memory with coalesced loads,
//     transposed so that element e of every matrix forms one contiguous row
//     (thread t's copy sits at row e, column t: bank-conflict free).  Each
//     thread then runs Eqs. 3-4 and the Sec. IV.A recurrence on its own
//     matrix, either from registers (small N) or in place in shared memory.
//   warp kernels (one matrix per warp, runtime N): the matrix sits in shared
//     memory as a padded dense square; lanes own columns and the column dot
//     products of Eqs. 3-4 and of the inverse run across lanes.
#pragma once

#include "common.cuh"

namespace cholinv {

// Arguments common to every batched kernel.
struct BatchParams {
    int32_t batch;             // matrices in the call
    const int32_t* n;          // per-matrix order (NULL: uniform max_n)
    const int64_t* off;        // per-matrix element offset (NULL: contiguous)
    int32_t max_n;
    int32_t layout;            // 0 dense, 1 packed upper
    int32_t fill_lower;        // dense X: also write the lower half
    int32_t want_inv;          // 0: factor only (R), 1: inverse (X, optional R)
    const void* A;
    void* R;                   // may be NULL when want_inv
    void* X;
    int32_t* info;             // may be NULL
    const int32_t* cls_count;  // per-class counts (bucketed batches) or NULL
    const int32_t* cls_start;  // per-class start in perm
    const int32_t* perm;       // matrix indices sorted by class
    int* err;                  // device error word
    int32_t flags;             // CHOL_FLAG_*
    uint64_t order_mask[2];    // bit c: order c may occur (bucketing rejects the others)
    unsigned long long* redo_count;  // matrices redone with FP64 pivots (CHOL_FLAG_PIVOT64_AUTO)
    int32_t aligned16;         // A, R and X all start on 16-byte boundaries (16-byte copies allowed)
};

// CHOL_FLAG_PIVOT64_AUTO: a matrix whose FP32 pass saw cancellation in Eq. 3
// (t_i < 2^-10 a_ii at some row, or a non-positive or non-finite t_i) is
// marked with this info value, nothing of it is stored, and a second pass
// (k_redo) factors and inverts it again with the sum of Eq. 3 accumulated in
// FP64.  t_i >= lambda_min(A) and a_ii <= lambda_max(A), so a matrix with
// kappa_2(A) < 2^10 is never marked.
constexpr int kInfoRedo = -2;

// Size classes of the bucketing (orders 0..71).
constexpr int kClasses = 72;
template <typename R> CHOL_D bool pivot_cancels(R t, R aii) { return !(t >= aii * R(0.0009765625)); }

// Arguments of the MMSE-filter kernels (mmse.cu): H_b is m_b x n_b
// row-major at element hoff[b] (NULL: b * max_m * max_n); W_b = X_b H_b^* is
// n_b x m_b row-major at woff[b] (NULL: b * max_n * max_m); A and X are the
// packed Gram matrices and their inverses at b * T(max_n) in the workspace.
struct MmseParams {
    int32_t batch;
    const int32_t* n;
    const int32_t* m;
    const int64_t* hoff;
    const int64_t* woff;
    int32_t max_n, max_m;
    const void* H;
    void* A;
    void* X;
    void* W;
    const int32_t* info;
};

// Arguments of the adjoint kernel.
struct BwdParams {
    int32_t batch;
    const int32_t* n;          // per-matrix order (NULL: uniform max_n)
    const int64_t* off;        // element offsets of G and dA (dense layout)
    const int64_t* xoff;       // element offsets of X (its own layout)
    int32_t max_n;
    int32_t layout;            // layout of X
    const void* X;
    const void* G;
    void* dA;
    int32_t flags;             // CHOL_FLAG_GRAD_UPPER selects the upper-parameter form
};

// Eq. 3's argument with its sum accumulated in FP64 (the sum of |r_ki|^2 over
// FP32 values is formed from exact FP64 products); used for FP32 value types
// under CHOL_FLAG_PIVOT64 to avoid losing the pivot to cancellation.
template <typename V>
CHOL_D double pivot64_term(V v) {
    if constexpr (traits<V>::cplx) return (double)v.re * (double)v.re + (double)v.im * (double)v.im;
    else return (double)v * (double)v;
}

// Matrix index of the k-th member of class N, and its element offset.
CHOL_D int64_t member_index(const BatchParams& p, int N, int k) {
    if (p.perm) return p.perm[p.cls_start[N] + k];
    return k;
}
CHOL_D int64_t matrix_offset(const BatchParams& p, int N, int64_t b) {
    (void)N;
    if (p.off) return p.off[b];
    // without offsets every matrix takes the room of one of order max_n
    return b * (p.layout ? tri64(p.max_n) : (int64_t)p.max_n * p.max_n);
}
CHOL_D int class_count(const BatchParams& p, int N) {
    return p.cls_count ? p.cls_count[N] : p.batch;
}

// ---------------------------------------------------------------------------
// The method on one matrix held in packed-upper order, N compile-time.
// Acc::at(e) returns a reference to element e (registers or shared memory).
// ---------------------------------------------------------------------------
// (Loops below run over fixed trip counts with compile-time guards: with
// bounds that depend on an outer index the front end leaves a register array
// in local memory.)
// LDL: the LDL form of Sec. II.A (Eqs. 9-11) instead: R unit upper, d_i on
// its diagonal, d_i = a_ii - sum_k d_k |r_ki|^2 and
// r_ij = (a_ij - sum_k conj(r_ki) d_k r_kj) / d_i; dinv[i] = 1/d_i.
// P64: Eq. 3 accumulated in FP64 (CHOL_FLAG_PIVOT64; FP32 value types), a
// compile-time choice so that the default kernels carry no branch for it.
template <typename V, int N, bool LDL = false, bool P64 = false, class Acc>
CHOL_D int factor_unrolled(Acc& m, typename traits<V>::real (&dinv)[N > 0 ? N : 1], bool gate = false) {
    using R = typename traits<V>::real;
    int info = 0;
    bool redo = false;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        V col[N > 0 ? N : 1];  // column i of R above the diagonal: r_ki, k < i (LDL: d_k r_ki)
#pragma unroll
        for (int k = 0; k < N; ++k)
            if (k < i) col[k] = m.at(pidx(N, k, i));
        // Eq. 3
        R t = re_of(m.at(pidx(N, i, i)));
        R rii, inv;
        if constexpr (LDL) {
            // Eq. 10: d_i; column i scaled by d_k for Eq. 11
#pragma unroll
            for (int k = 0; k < N; ++k) {
                if (k < i) {
                    const V w = scale_v(col[k], re_of(m.at(pidx(N, k, k))));
                    t = fma_re_conjb(-w, col[k], t);
                    col[k] = w;
                }
            }
            if (info == 0 && !pivot_ok(t)) info = i + 1;
            rii = t;
            inv = R(1) / t;
        } else if constexpr (sizeof(R) == 4 && P64) {
            double td = (double)t;
#pragma unroll
            for (int k = 0; k < N; ++k)
                if (k < i) td -= pivot64_term(col[k]);
            t = (R)td;
            pivot_root64(td, rii, inv);
            if (info == 0 && !pivot_ok(td)) info = i + 1;
        } else {
            const R aii = t;
#pragma unroll
            for (int k = 0; k < N; ++k)
                if (k < i) t = fnma_abs2(col[k], t);
            if (gate && pivot_cancels(t, aii)) redo = true;
            if (info == 0 && !pivot_ok(t)) info = i + 1;
            pivot_root(t, rii, inv);
        }
        dinv[i] = inv;
        m.at(pidx(N, i, i)) = from_real<V>(rii);
        // Eq. 4
#pragma unroll
        for (int j = 0; j < N; ++j) {
            if (j > i) {
                V s = m.at(pidx(N, i, j));
#pragma unroll
                for (int k = 0; k < N; ++k)
                    if (k < i) s = fnma_conj(col[k], m.at(pidx(N, k, j)), s);
                m.at(pidx(N, i, j)) = scale_v(s, inv);
            }
        }
    }
    return redo ? kInfoRedo : info;
}

// Proposed inverse (Eqs. 20-24) in place over R: row i of R is read into
// registers, then replaced by row i of X.  Each stored x_km (i < k <= m) is
// read once and feeds two sums: x_im (term k, r_ik x_km) and, when k < m,
// x_ik (term m, r_im conj(x_km)).  For every target the terms still arrive
// with k ascending, the order of the definition.  LDL: the form of Sec.
// IV.B (Eqs. 25-29) over a unit upper R, x_ij = -sum r_ik x~_kj and
// x_ii = 1/d_i - sum r_ik conj(x_ik).
template <typename V, int N, bool LDL = false, class Acc>
CHOL_D void inverse_unrolled(Acc& m, const typename traits<V>::real (&dinv)[N > 0 ? N : 1]) {
    using R = typename traits<V>::real;
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {
        V row[N > 0 ? N : 1];
        V acc[N > 0 ? N : 1];
#pragma unroll
        for (int k = 0; k < N; ++k)
            if (k > i) { row[k] = m.at(pidx(N, i, k)); acc[k] = zero_v<V>(); }
#pragma unroll
        for (int k = 0; k < N; ++k) {
            if (k > i) {
#pragma unroll
                for (int c = 0; c < N; ++c) {
                    if (c >= k) {
                        V v = m.at(pidx(N, k, c));
                        acc[c] = fma_v(row[k], v, acc[c]);
                        if (c > k) acc[k] = fma_conjb(row[c], v, acc[k]);
                    }
                }
            }
        }
        const R inv = dinv[i];
        R sd = R(0);
#pragma unroll
        for (int j = 0; j < N; ++j) {
            if (j > i) {
                V x = LDL ? -acc[j] : scale_v(acc[j], -inv);
                m.at(pidx(N, i, j)) = x;
                sd = fma_re_conjb(row[j], x, sd);
            }
        }
        m.at(pidx(N, i, i)) = from_real<V>(LDL ? inv - sd : (inv - sd) * inv);
    }
}

// ---------------------------------------------------------------------------
// Asynchronous global -> shared copies (cp.async; sm_80+ PTX).
// ---------------------------------------------------------------------------
CHOL_D unsigned smem_u32(const void* p) { return static_cast<unsigned>(__cvta_generic_to_shared(p)); }

template <int BYTES>
CHOL_D void cp_async(void* dst_smem, const void* src) {
    if constexpr (BYTES == 16) {
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst_smem)), "l"(src) : "memory");
    } else {
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(smem_u32(dst_smem)), "l"(src), "n"(BYTES)
                     : "memory");
    }
}
CHOL_D void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int PENDING>
CHOL_D void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(PENDING) : "memory"); }

// ---------------------------------------------------------------------------
// Lane kernel layout.  A CTA handles THREADS matrices per chunk.  Shared
// memory holds each matrix's packed triangle in 16-byte units (U elements
// per unit); unit u of the matrix of thread q sits at [u][q] (row stride
// LD = THREADS + 1 units), so a warp reading unit u of its 32 matrices, or a
// loader writing consecutive units of one matrix, touches distinct banks.
// ---------------------------------------------------------------------------
template <typename V, int N>
struct LaneCfg {
    static constexpr int TN = tri(N);
    static constexpr int U = 16 / (int)sizeof(V);      // elements per 16-byte unit
    static constexpr int NU = (TN + U - 1) / U;        // units per matrix
    // Registers hold the whole matrix when its packed triangle takes at most
    // 144 32-bit words; larger matrices are worked in place in shared memory.
    static constexpr bool REGS = TN * traits<V>::words <= 144;
    static constexpr int UNIT_BYTES = 16;
    static constexpr int bytes_per_matrix = NU * UNIT_BYTES;
    // register-resident kernels double-buffer (load chunk k+1 while computing k)
    static constexpr int NBUF = REGS ? 2 : 1;
    static constexpr int THREADS = bytes_per_matrix * 128 * NBUF <= 98304 ? 128
                                 : bytes_per_matrix * 64 * NBUF <= 98304 ? 64 : 32;
    static constexpr int LD = THREADS + 1;             // units per shared row
    static constexpr size_t BUF_BYTES = (size_t)NU * LD * UNIT_BYTES;
    static constexpr size_t SMEM = NBUF * BUF_BYTES + (size_t)THREADS * (NBUF * sizeof(int64_t) + sizeof(int)) +
                                   2 * (size_t)TN + 16;
};

template <typename V, int N>
struct UnitRef {  // element e of the matrix of thread q inside a unit buffer
    static CHOL_D V& at(uint4* buf, int q, int e) {
        constexpr int U = LaneCfg<V, N>::U;
        constexpr int LD = LaneCfg<V, N>::LD;
        return reinterpret_cast<V*>(buf + (e / U) * LD + q)[e % U];
    }
};

template <typename V, int TN>
struct RegMat {
    V a[TN];
    CHOL_D V& at(int e) { return a[e]; }
};

template <typename V, int N>
struct SmemMat {
    uint4* buf;
    int q;
    CHOL_D V& at(int e) { return UnitRef<V, N>::at(buf, q, e); }
};

// Stage the chunk's matrices into a unit buffer with cp.async (not waited on).
// vec: every matrix starts on a 16-byte boundary and the layout is packed, so
// whole units are copied; otherwise element by element (dense layout or
// unaligned offsets).
template <typename V, int N>
CHOL_D void lane_stage(const BatchParams& p, const V* A, uint4* buf, const int64_t* s_off, const uint8_t* s_i,
                       const uint8_t* s_j, int m, bool vec) {
    using C = LaneCfg<V, N>;
    const int t = threadIdx.x;
    if (vec) {
        for (int f = t; f < m * C::NU; f += C::THREADS) {
            const int q = f / C::NU, u = f - q * C::NU;
            const V* src = A + s_off[q] + u * C::U;
            uint4* dst = buf + u * C::LD + q;
            if ((u + 1) * C::U <= C::TN) {
                cp_async<16>(dst, src);
            } else {
#pragma unroll
                for (int r = 0; r < C::U; ++r)
                    if (u * C::U + r < C::TN) cp_async<(int)sizeof(V)>(reinterpret_cast<V*>(dst) + r, src + r);
            }
        }
    } else {
        for (int f = t; f < m * C::TN; f += C::THREADS) {
            const int q = f / C::TN, e = f - q * C::TN;
            const int64_t g = p.layout ? (int64_t)e : (int64_t)s_i[e] * N + s_j[e];
            cp_async<(int)sizeof(V)>(&UnitRef<V, N>::at(buf, q, e), A + s_off[q] + g);
        }
    }
    cp_async_commit();
}

// Write the chunk's results (X, or R when factoring) from a unit buffer.
// GATE: matrices marked kInfoRedo are skipped (CHOL_FLAG_PIVOT64_AUTO).
template <typename V, int N, bool GATE = false>
CHOL_D void lane_store(const BatchParams& p, V* out, uint4* buf, const int64_t* s_off, const int* s_info,
                       const uint8_t* s_i, const uint8_t* s_j, int m, bool vec, bool is_factor, bool fill_lower) {
    using C = LaneCfg<V, N>;
    const int t = threadIdx.x;
    if (vec) {
        for (int f = t; f < m * C::NU; f += C::THREADS) {
            const int q = f / C::NU, u = f - q * C::NU;
            if constexpr (GATE)
                if (s_info[q] == kInfoRedo) continue;  // left to the FP64-pivot pass
            V* dst = out + s_off[q] + u * C::U;
            uint4 v = buf[u * C::LD + q];
            if (s_info[q] != 0) {
                const V qn = nan_v<V>();
#pragma unroll
                for (int r = 0; r < C::U; ++r) reinterpret_cast<V*>(&v)[r] = qn;
            }
            if ((u + 1) * C::U <= C::TN) {
                *reinterpret_cast<uint4*>(dst) = v;
            } else {
#pragma unroll
                for (int r = 0; r < C::U; ++r)
                    if (u * C::U + r < C::TN) dst[r] = reinterpret_cast<V*>(&v)[r];
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
            const V v = bad ? nan_v<V>() : UnitRef<V, N>::at(buf, q, e);
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

// ---------------------------------------------------------------------------
// Lane kernel: one matrix per thread.
// ---------------------------------------------------------------------------
// GATE: CHOL_FLAG_PIVOT64_AUTO's cancellation test (FP32 value types only).
// LDL: the LDL form (CHOL_FLAG_LDL).  P64: FP64 pivots (CHOL_FLAG_PIVOT64).
template <typename V, int N, bool GATE = false, bool LDL = false, bool P64 = false>
__global__ void __launch_bounds__(LaneCfg<V, N>::THREADS)
k_lane(BatchParams p) {
    using C = LaneCfg<V, N>;
    constexpr int THREADS = C::THREADS;
    constexpr int TN = C::TN;
    using R = typename traits<V>::real;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint4* bufs = reinterpret_cast<uint4*>(smem_raw);                                // NBUF x [NU][LD] units
    int64_t* s_offs = reinterpret_cast<int64_t*>(smem_raw + C::NBUF * C::BUF_BYTES);  // NBUF x [THREADS]
    int* s_info = reinterpret_cast<int*>(s_offs + C::NBUF * THREADS);                 // [THREADS]
    uint8_t* s_i = reinterpret_cast<uint8_t*>(s_info + THREADS);                      // [TN] row of element e
    uint8_t* s_j = s_i + TN;                                                          // [TN] column of element e

    const int t = threadIdx.x;
    for (int e = t; e < TN; e += THREADS) {
        int i = 0;
        while (pidx(N, i + 1, i + 1) <= e && i + 1 < N) ++i;
        s_i[e] = (uint8_t)i;
        s_j[e] = (uint8_t)(e - pidx(N, i, i) + i);
    }
    const int count = class_count(p, N);
    const int nchunks = (count + THREADS - 1) / THREADS;
    const V* A = static_cast<const V*>(p.A);
    V* Xo = static_cast<V*>(p.X);
    V* Ro = static_cast<V*>(p.R);
    const bool store_R = p.R != nullptr && p.want_inv;
    constexpr bool gate = GATE;

    // Offsets of a chunk's matrices into s_off; returns (CTA-uniformly)
    // whether whole 16-byte units can be copied.
    auto chunk_offsets = [&](int chunk, int m, int64_t* s_off) {
        int ok = 1;
        if (t < m) {
            const int64_t b = member_index(p, N, chunk * THREADS + t);
            const int64_t o = matrix_offset(p, N, b);
            s_off[t] = o;
            ok = (o % C::U) == 0;
        }
        return __syncthreads_and(ok) != 0 && p.layout == 1 && p.aligned16;
    };

    if constexpr (C::REGS) {
        // ---- register-resident: double-buffered, chunk k+1 loads while k computes
        int chunk = blockIdx.x;
        if (chunk >= nchunks) return;
        int m = min(THREADS, count - chunk * THREADS);
        bool vec = chunk_offsets(chunk, m, s_offs);
        int cur = 0;
        lane_stage<V, N>(p, A, bufs, s_offs, s_i, s_j, m, vec);
        for (; chunk < nchunks; chunk += gridDim.x) {
            uint4* buf = bufs + cur * (C::BUF_BYTES / 16);
            int64_t* s_off = s_offs + cur * THREADS;
            cp_async_wait<0>();
            __syncthreads();
            RegMat<V, TN> r;
#pragma unroll
            for (int e = 0; e < TN; ++e) r.a[e] = UnitRef<V, N>::at(buf, t, e);
            const int64_t my_off = t < m ? s_off[t] : 0;
            // prefetch the next chunk into the other buffer
            const int next = chunk + gridDim.x;
            int m_next = 0;
            bool vec_next = false;
            if (next < nchunks) {
                m_next = min(THREADS, count - next * THREADS);
                vec_next = chunk_offsets(next, m_next, s_offs + (cur ^ 1) * THREADS);
                lane_stage<V, N>(p, A, bufs + (cur ^ 1) * (C::BUF_BYTES / 16), s_offs + (cur ^ 1) * THREADS, s_i,
                                 s_j, m_next, vec_next);
            }
            int info = 0;
            R dinv[N];
            if (t < m) {
                info = factor_unrolled<V, N, LDL, P64>(r, dinv, gate);
                if (store_R && (!GATE || info != kInfoRedo)) {
#pragma unroll
                    for (int e = 0; e < TN; ++e) {
                        const int64_t g = p.layout ? (int64_t)e : (int64_t)s_i[e] * N + s_j[e];
                        Ro[my_off + g] = info ? nan_v<V>() : r.a[e];
                    }
                    if (!p.layout) {
#pragma unroll
                        for (int e = 0; e < TN; ++e)
                            if (s_i[e] != s_j[e])
                                Ro[my_off + (int64_t)s_j[e] * N + s_i[e]] = info ? nan_v<V>() : zero_v<V>();
                    }
                }
                if (p.want_inv) inverse_unrolled<V, N, LDL>(r, dinv);
#pragma unroll
                for (int e = 0; e < TN; ++e) UnitRef<V, N>::at(buf, t, e) = r.a[e];
                s_info[t] = info;
            }
            __syncthreads();
            lane_store<V, N, GATE>(p, p.want_inv ? Xo : Ro, buf, s_off, s_info, s_i, s_j, m, vec, !p.want_inv,
                             p.fill_lower != 0);
            if (p.info)
                for (int q = t; q < m; q += THREADS) p.info[member_index(p, N, chunk * THREADS + q)] = s_info[q];
            __syncthreads();
            m = m_next;
            vec = vec_next;
            cur ^= 1;
        }
    } else {
        // ---- shared-memory-resident: one buffer, the method runs in place
        uint4* buf = bufs;
        int64_t* s_off = s_offs;
        for (int chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
            const int m = min(THREADS, count - chunk * THREADS);
            const bool vec = chunk_offsets(chunk, m, s_off);
            lane_stage<V, N>(p, A, buf, s_off, s_i, s_j, m, vec);
            cp_async_wait<0>();
            __syncthreads();
            int info = 0;
            R dinv[N];
            SmemMat<V, N> sm{buf, t};
            if (t < m) info = factor_unrolled<V, N, LDL, P64>(sm, dinv, gate);
            if (t < m) s_info[t] = info;
            if (store_R) {
                __syncthreads();
                lane_store<V, N, GATE>(p, Ro, buf, s_off, s_info, s_i, s_j, m, vec, true, false);
                __syncthreads();
            }
            if (p.want_inv && t < m) inverse_unrolled<V, N, LDL>(sm, dinv);
            __syncthreads();
            lane_store<V, N, GATE>(p, p.want_inv ? Xo : Ro, buf, s_off, s_info, s_i, s_j, m, vec, !p.want_inv,
                             p.fill_lower != 0);
            if (p.info)
                for (int q = t; q < m; q += THREADS) p.info[member_index(p, N, chunk * THREADS + q)] = s_info[q];
            __syncthreads();
        }
    }
}

// Shared-memory elements of one warp of the warp kernel: the padded square
// (N x (N+1)), and a second one for the comparison methods' B or M.
CHOL_HD size_t warp_elems(const BatchParams& p, int N) {
    const size_t sq = (size_t)N * (N + 1);
    return (p.flags & (CHOL_FLAG_METHOD_ES | CHOL_FLAG_METHOD_TMO)) ? 2 * sq : sq;
}

// ---------------------------------------------------------------------------
// Warp-wide staging of one matrix from global into shared memory.
// ---------------------------------------------------------------------------
// f(e, src[e]) for e = 0..count-1 over the 32 lanes of a warp, each lane
// issuing eight loads before it hands any on: a matrix costs a few memory
// round trips instead of one per element a lane takes.
template <typename V, class F>
CHOL_D void warp_gather(const V* __restrict__ src, int count, int lane, F&& f) {
    constexpr int U = 8;
#pragma unroll 1
    for (int e0 = 0; e0 < count; e0 += 32 * U) {
        V v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + u * 32 + lane;
            if (e < count) v[u] = src[e];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + u * 32 + lane;
            if (e < count) f(e, v[u]);
        }
    }
}

// Row and column of element e of an order-n matrix stored dense (row-major)
// or packed (upper triangle by rows); dense elements below the diagonal
// come back with i > j.
CHOL_D void elem_rc(int layout, int n, int e, int& i, int& j) {
    if (layout) {
        tri_rc(n, e, i, j);
    } else {
        i = e / n;
        j = e - i * n;
    }
}

// f(i, j, element (i, j)) over a rows x cols matrix at src by one warp,
// lanes over the columns j = lane + 32 h (h < NS, so cols <= 32 NS), U rows
// a round with every load of the round in flight before any is handed on.
// UPPER: an order-rows matrix's upper triangle only (j >= i), stored dense
// or packed (`layout`); else a dense row-major matrix in full.  No index
// needs a division, but lanes beyond `cols` idle: for matrices of order
// near 32 or 64 (warp_gather keeps every lane busy for smaller ones).
template <bool UPPER, int NS = 2, int U = 4, typename V, class F>
CHOL_D void warp_rows(const V* __restrict__ src, int rows, int cols, int layout, int lane, F&& f) {
#pragma unroll 1
    for (int i0 = 0; i0 < rows; i0 += U) {
        V v[U][NS];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int h = 0; h < NS; ++h) {
                const int i = i0 + u, j = lane + 32 * h;
                if (i < rows && j < cols && (!UPPER || j >= i))
                    v[u][h] = src[(UPPER && layout) ? pidx(cols, i, j) : i * cols + j];
            }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int h = 0; h < NS; ++h) {
                const int i = i0 + u, j = lane + 32 * h;
                if (i < rows && j < cols && (!UPPER || j >= i)) f(i, j, v[u][h]);
            }
    }
}

// The upper triangle of the order-n matrix at src (dense or packed) into the
// square S (row stride ld) in full: mirrored (conjugated), diagonal real.
template <typename V>
CHOL_D void stage_hermitian(const V* __restrict__ src, int n, int layout, V* S, int ld, int lane) {
    warp_gather(src, layout ? n * (n + 1) / 2 : n * n, lane, [&](int e, V v) {
        int i, j;
        elem_rc(layout, n, e, i, j);
        if (i <= j) {
            const V x = (i == j) ? from_real<V>(re_of(v)) : v;
            S[i * ld + j] = x;
            S[j * ld + i] = conj_v(x);
        }
    });
}

// One warp's asynchronous copy (cp.async; complete after cp_async_wait) of
// `count` elements from global src to shared dst: 16-byte units when both
// ends are 16-byte aligned and the size is a multiple of 16, else 4-byte
// units (every element type here is a whole number of aligned words).
template <typename V>
CHOL_D void warp_copy_async(V* dst, const V* src, int count, int lane) {
    const int bytes = count * (int)sizeof(V);
    char* d = reinterpret_cast<char*>(dst);
    const char* s = reinterpret_cast<const char*>(src);
    if (((reinterpret_cast<uintptr_t>(d) | reinterpret_cast<uintptr_t>(s)) % 16) == 0 && bytes % 16 == 0) {
        for (int k = lane; k < bytes / 16; k += 32) cp_async<16>(d + 16 * k, s + 16 * k);
    } else {
        for (int k = lane; k < bytes / 4; k += 32) cp_async<4>(d + 4 * k, s + 4 * k);
    }
}

// The upper triangle of an order-n matrix held as stored (dense or packed)
// in shared memory into the square S (row stride ld) in full: mirrored
// (conjugated), diagonal real.
template <typename V>
CHOL_D void unpack_hermitian(const V* raw, int n, int layout, V* S, int ld, int lane) {
    const int count = layout ? n * (n + 1) / 2 : n * n;
    for (int e = lane; e < count; e += 32) {
        int i, j;
        elem_rc(layout, n, e, i, j);
        if (i <= j) {
            const V x = (i == j) ? from_real<V>(re_of(raw[e])) : raw[e];
            S[i * ld + j] = x;
            S[j * ld + i] = conj_v(x);
        }
    }
}

// ---------------------------------------------------------------------------
// Warp kernel: one matrix per warp, runtime order N (<= 64), lanes own the
// columns j = lane and j = lane + 32.  The matrix is a padded dense square
// in shared memory (row stride N+1).
// ---------------------------------------------------------------------------
// One matrix (index b, element offset o, order N) on one warp; S holds
// N x (N+1) elements.  pivot64: Eq. 3 accumulated in FP64 (FP32 value
// types); gate: mark the matrix for the FP64-pivot pass on cancellation.
template <typename V>
CHOL_D void warp_one(const BatchParams& p, int N, int64_t b, int64_t o, V* S, int lane, bool pivot64, bool gate) {
    using R = typename traits<V>::real;
    const int LD = N + 1;
    const V* A = static_cast<const V*>(p.A);
    V* Xo = static_cast<V*>(p.X);
    V* Ro = static_cast<V*>(p.R);
    // load the upper triangle
    warp_gather(A + o, p.layout ? tri(N) : N * N, lane, [&](int e, V v) {
        int i, j;
        elem_rc(p.layout, N, e, i, j);
        if (i <= j) S[i * LD + j] = v;
    });
    __syncwarp();
    // ---- factor, Eqs. 3-4, row by row; with CHOL_FLAG_LDL the LDL form of
    // Sec. II.A (Eqs. 9-11): d_i = a_ii - sum |r_ki|^2 d_k and
    // r_ij = (a_ij - sum conj(r_ki) d_k r_kj) / d_i, R unit upper, d_i kept
    // on R's diagonal
    const bool ldl = (p.flags & CHOL_FLAG_LDL) != 0;
    int info = 0;
    bool redo = false;
    for (int i = 0; i < N; ++i) {
        const R aii = re_of(S[i * LD + i]);  // read before this row is written
        V s0 = zero_v<V>(), s1 = zero_v<V>();
        const int j0 = lane, j1 = lane + 32;
        if (j0 >= i && j0 < N) {
            s0 = S[i * LD + j0];
            for (int k = 0; k < i; ++k) {
                const V rki = ldl ? scale_v(S[k * LD + i], re_of(S[k * LD + k])) : S[k * LD + i];
                s0 = fnma_conj(rki, S[k * LD + j0], s0);
            }
        }
        if (j1 >= i && j1 < N) {
            s1 = S[i * LD + j1];
            for (int k = 0; k < i; ++k) {
                const V rki = ldl ? scale_v(S[k * LD + i], re_of(S[k * LD + k])) : S[k * LD + i];
                s1 = fnma_conj(rki, S[k * LD + j1], s1);
            }
        }
        // pivot: column i lives in lane i & 31, slot i >> 5
        R tsrc = re_of((i < 32) ? s0 : s1);
        R tt = __shfl_sync(0xffffffffu, tsrc, i & 31);
        R rii, inv;
        if (ldl) {
            if (info == 0 && !pivot_ok(tt)) info = i + 1;
            rii = tt;  // d_i, stored on the diagonal
            inv = R(1) / tt;
        } else if (sizeof(R) == 4 && pivot64) {
            double td = (double)aii;
            for (int k = 0; k < i; ++k) td -= pivot64_term(S[k * LD + i]);
            if (info == 0 && !pivot_ok(td)) info = i + 1;
            pivot_root64(td, rii, inv);
        } else {
            if (gate && pivot_cancels(tt, aii)) redo = true;
            if (info == 0 && !pivot_ok(tt)) info = i + 1;
            pivot_root(tt, rii, inv);
        }
        if (j0 > i && j0 < N) S[i * LD + j0] = scale_v(s0, inv);
        if (j1 > i && j1 < N) S[i * LD + j1] = scale_v(s1, inv);
        if (lane == (i & 31)) S[i * LD + i] = from_real<V>(rii);
        __syncwarp();
    }
    if (redo) info = kInfoRedo;  // nothing stored: the FP64-pivot pass redoes this matrix
    if (p.R && !redo) {
        // store R (dense: zero strictly lower part)
        for (int i = 0; i < N; ++i)
            for (int j = lane; j < N; j += 32) {
                if (j >= i) {
                    const int64_t g = p.layout ? (int64_t)pidx(N, i, j) : (int64_t)i * N + j;
                    Ro[o + g] = info ? nan_v<V>() : S[i * LD + j];
                } else if (!p.layout) {
                    Ro[o + (int64_t)i * N + j] = info ? nan_v<V>() : zero_v<V>();
                }
            }
    }
    const int method = (p.flags & CHOL_FLAG_METHOD_ES) ? 1 : (p.flags & CHOL_FLAG_METHOD_TMO) ? 2 : 0;
    if (p.want_inv && !redo && method == 1) {
        // ---- existing method "Equation Solving" (Sec. III.A, Eq. 15): for
        // every column j the forward solve R^* b = e_j (b_k = 0 for k < j;
        // lanes own right-hand sides), then the back substitution
        // x_ij = (b_i - sum_{k>i} r_ik x~_kj) / r_ii for i <= j, rows N..1,
        // with b_i taken from the forward solve.  B (row j = b for e_j) sits
        // after the matrix in this warp's shared memory.
        V* B = S + (size_t)N * LD;
        for (int jj = lane; jj < N; jj += 32) {
            for (int k = jj; k < N; ++k) {
                V t = (k == jj) ? from_real<V>(R(1)) : zero_v<V>();
                for (int l = jj; l < k; ++l) t = fnma_conj(S[l * LD + k], B[jj * LD + l], t);
                B[jj * LD + k] = scale_v(t, R(1) / re_of(S[k * LD + k]));
            }
        }
        __syncwarp();
        for (int i = N - 1; i >= 0; --i) {
            const R inv = R(1) / re_of(S[i * LD + i]);
            V x[2] = {zero_v<V>(), zero_v<V>()};
            R sd = R(0);
            for (int h = 0; h < 2; ++h) {
                const int j = lane + 32 * h;
                if (j > i && j < N) {
                    V a = zero_v<V>();  // b_i = 0 for i < j
                    for (int k = i + 1; k < N; ++k) {
                        const V xt = (k <= j) ? S[k * LD + j] : conj_v(S[j * LD + k]);
                        a = fma_v(S[i * LD + k], xt, a);
                    }
                    x[h] = scale_v(a, -inv);
                    sd = fma_re_conjb(S[i * LD + j], x[h], sd);
                }
            }
            __syncwarp();
            for (int h = 0; h < 2; ++h) {
                const int j = lane + 32 * h;
                if (j > i && j < N) S[i * LD + j] = x[h];
            }
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) sd += __shfl_xor_sync(0xffffffffu, sd, d);
            __syncwarp();
            // the diagonal: (b_i - sum_k r_ik x~_ki) / r_ii with b_i = B[i][i] from the forward solve
            if (lane == 0) S[i * LD + i] = from_real<V>((re_of(B[i * LD + i]) - sd) * inv);
            __syncwarp();
        }
    } else if (p.want_inv && !redo && method == 2) {
        // ---- existing method "Triangular Matrix Operations" (Sec. III.B,
        // Eqs. 16-19): M = R^{-1} column by column from R m_i = e_i (lanes
        // own columns), then the upper half of X = M M^*,
        // x_ij = sum_{l>=j} m_il conj(m_jl).  M sits after the matrix.
        V* Mm = S + (size_t)N * LD;
        for (int ii = lane; ii < N; ii += 32) {
            Mm[ii * LD + ii] = from_real<V>(R(1) / re_of(S[ii * LD + ii]));
            for (int k = ii - 1; k >= 0; --k) {
                V t = zero_v<V>();
                for (int l = k + 1; l <= ii; ++l) t = fma_v(S[k * LD + l], Mm[l * LD + ii], t);
                Mm[k * LD + ii] = scale_v(t, -R(1) / re_of(S[k * LD + k]));
            }
        }
        __syncwarp();
        for (int jj = lane; jj < N; jj += 32) {
            for (int i = 0; i <= jj; ++i) {
                V t = zero_v<V>();
                for (int l = jj; l < N; ++l) t = fma_conjb(Mm[i * LD + l], Mm[jj * LD + l], t);
                S[i * LD + jj] = (i == jj) ? from_real<V>(re_of(t)) : t;
            }
        }
        __syncwarp();
    } else if (p.want_inv && !redo) {
        // ---- proposed inverse, rows N..1
        for (int i = N - 1; i >= 0; --i) {
            const int j0 = lane, j1 = lane + 32;
            V a0 = zero_v<V>(), a1 = zero_v<V>();
            V r0 = zero_v<V>(), r1 = zero_v<V>();
            if (j0 > i && j0 < N) {
                r0 = S[i * LD + j0];
                for (int k = i + 1; k < N; ++k) {
                    V xt = (k <= j0) ? S[k * LD + j0] : conj_v(S[j0 * LD + k]);
                    a0 = fma_v(S[i * LD + k], xt, a0);
                }
            }
            if (j1 > i && j1 < N) {
                r1 = S[i * LD + j1];
                for (int k = i + 1; k < N; ++k) {
                    V xt = (k <= j1) ? S[k * LD + j1] : conj_v(S[j1 * LD + k]);
                    a1 = fma_v(S[i * LD + k], xt, a1);
                }
            }
            // 1/r_ii, or 1/d_i in the LDL form (Sec. IV.B, Eqs. 25-29: R unit
            // upper, s~_ii = 1/d_i, so x_ij = -sum r_ik x~_kj and
            // x_ii = 1/d_i - sum r_ik conj(x_ik))
            const R inv = R(1) / re_of(S[i * LD + i]);
            const R xs = ldl ? R(-1) : -inv;
            __syncwarp();
            R sd = R(0);
            if (j0 > i && j0 < N) { V x = scale_v(a0, xs); S[i * LD + j0] = x; sd = fma_re_conjb(r0, x, sd); }
            if (j1 > i && j1 < N) { V x = scale_v(a1, xs); S[i * LD + j1] = x; sd = fma_re_conjb(r1, x, sd); }
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) sd += __shfl_xor_sync(0xffffffffu, sd, d);
            __syncwarp();
            if (lane == 0) S[i * LD + i] = from_real<V>(ldl ? inv - sd : (inv - sd) * inv);
            __syncwarp();
        }
    }
    if (p.want_inv && !redo) {
        // store X
        for (int i = 0; i < N; ++i)
            for (int j = i + lane; j < N; j += 32) {
                V v = info ? nan_v<V>() : S[i * LD + j];
                if (p.layout) {
                    Xo[o + pidx(N, i, j)] = v;
                } else {
                    Xo[o + (int64_t)i * N + j] = v;
                    if (p.fill_lower && j > i) Xo[o + (int64_t)j * N + i] = conj_v(v);
                }
            }
    }
    if (p.info && lane == 0) p.info[b] = info;
    __syncwarp();
}

template <typename V>
__global__ void k_warp(BatchParams p, int N, int warps_per_cta) {
    using R = typename traits<V>::real;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    V* S = reinterpret_cast<V*>(smem_raw) + (size_t)w * warp_elems(p, N);
    const int count = class_count(p, N);
    const bool pivot64 = (p.flags & CHOL_FLAG_PIVOT64) != 0;
    const bool gate = sizeof(R) == 4 && (p.flags & CHOL_FLAG_PIVOT64_AUTO) && !pivot64;
    for (int k0 = blockIdx.x * warps_per_cta + w; k0 < count; k0 += gridDim.x * warps_per_cta) {
        const int64_t b = member_index(p, N, k0);
        warp_one<V>(p, N, b, matrix_offset(p, N, b), S, lane, pivot64, gate);
    }
}

// The FP64-pivot pass of CHOL_FLAG_PIVOT64_AUTO: every matrix of the batch
// whose info holds kInfoRedo is factored and inverted again, one per warp,
// with Eq. 3 accumulated in FP64; its outputs and info are written then.
// `smax` is the largest order of the call (shared memory per warp).
template <typename V>
__global__ void k_redo(BatchParams p, int smax, int warps_per_cta) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    V* S = reinterpret_cast<V*>(smem_raw) + (size_t)w * warp_elems(p, smax);
    for (int64_t b = (int64_t)blockIdx.x * warps_per_cta + w; b < p.batch; b += (int64_t)gridDim.x * warps_per_cta) {
        if (p.info[b] != kInfoRedo) continue;  // warp-uniform
        const int N = p.n ? p.n[b] : p.max_n;
        if (N < 1 || N > smax) continue;       // orders outside [1, max_n] were rejected by the bucketing
        warp_one<V>(p, N, b, matrix_offset(p, N, b), S, lane, true, false);
        if (lane == 0 && p.redo_count) atomicAdd(p.redo_count, 1ull);
    }
}

// One launch for the whole batch (CHOL_FLAG_SINGLE_LAUNCH): persistent
// warps take matrices one at a time from a device counter, largest orders
// first (the bucketing permutation read from its end), and run the
// one-matrix-per-warp body at each matrix's own order.  `smax` is the
// largest order of the call (shared memory per warp); *work is zero on
// entry.
template <typename V>
__global__ void k_warp_all(BatchParams p, int smax, int warps_per_cta, int* work) {
    using R = typename traits<V>::real;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    V* S = reinterpret_cast<V*>(smem_raw) + (size_t)w * warp_elems(p, smax);
    const bool pivot64 = (p.flags & CHOL_FLAG_PIVOT64) != 0;
    const bool gate = sizeof(R) == 4 && (p.flags & CHOL_FLAG_PIVOT64_AUTO) && !pivot64;
    const int64_t total = p.perm ? (int64_t)p.cls_start[kClasses - 1] + p.cls_count[kClasses - 1] : p.batch;
    for (;;) {
        int idx = 0;
        if (lane == 0) idx = atomicAdd(work, 1);
        idx = __shfl_sync(0xffffffffu, idx, 0);
        if (idx >= total) break;
        const int64_t b = p.perm ? (int64_t)p.perm[total - 1 - idx] : idx;
        const int N = p.n ? p.n[b] : p.max_n;
        warp_one<V>(p, N, b, matrix_offset(p, N, b), S, lane, pivot64, gate);
    }
}

// ---------------------------------------------------------------------------
// Size-class bucketing for batches with per-matrix orders.
// ws layout: counts[72] | starts[72] | cursor[72] | done | pad to 1024 B | perm[batch]
// ---------------------------------------------------------------------------

// Orders allowed by a mask (bit c of m[c / 64]).
CHOL_HD bool order_allowed(const uint64_t m0, const uint64_t m1, int c) {
    return c < 64 ? ((m0 >> c) & 1u) != 0 : ((m1 >> (c - 64)) & 1u) != 0;
}

__global__ void k_bucket_hist(int32_t batch, const int32_t* __restrict__ n, int32_t max_n, uint64_t m0, uint64_t m1,
                              int32_t* counts, int32_t* starts, int32_t* cursor, unsigned* done, int32_t* info,
                              int* err);
__global__ void k_bucket_scatter(int32_t batch, const int32_t* __restrict__ n, int32_t max_n, uint64_t m0,
                                 uint64_t m1, int32_t* cursor, int32_t* perm);

}  // namespace cholinv
