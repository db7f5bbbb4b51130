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
};

// Matrix index of the k-th member of class N, and its element offset.
CHOL_D int64_t member_index(const BatchParams& p, int N, int k) {
    if (p.perm) return p.perm[p.cls_start[N] + k];
    return k;
}
CHOL_D int64_t matrix_offset(const BatchParams& p, int N, int64_t b) {
    if (p.off) return p.off[b];
    return b * (p.layout ? tri64(N) : (int64_t)N * N);
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
template <typename V, int N, class Acc>
CHOL_D int factor_unrolled(Acc& m, typename traits<V>::real (&dinv)[N > 0 ? N : 1]) {
    using R = typename traits<V>::real;
    int info = 0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        V col[N > 0 ? N : 1];  // column i of R above the diagonal: r_ki, k < i
#pragma unroll
        for (int k = 0; k < N; ++k)
            if (k < i) col[k] = m.at(pidx(N, k, i));
        // Eq. 3
        R t = re_of(m.at(pidx(N, i, i)));
#pragma unroll
        for (int k = 0; k < N; ++k)
            if (k < i) t = fnma_abs2(col[k], t);
        if (info == 0 && !pivot_ok(t)) info = i + 1;
        R rii = sqrt(t);
        R inv = R(1) / rii;
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
    return info;
}

// Proposed inverse (Eqs. 20-24) in place over R: row i of R is read into
// registers, then replaced by row i of X.  Each stored x_km (i < k <= m) is
// read once and feeds two sums: x_im (term k, r_ik x_km) and, when k < m,
// x_ik (term m, r_im conj(x_km)).  For every target the terms still arrive
// with k ascending, the order of the definition.
template <typename V, int N, class Acc>
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
                V x = scale_v(acc[j], -inv);
                m.at(pidx(N, i, j)) = x;
                sd = fma_re_conjb(row[j], x, sd);
            }
        }
        m.at(pidx(N, i, i)) = from_real<V>((inv - sd) * inv);
    }
}

template <typename V, int TN>
struct RegMat {
    V a[TN];
    CHOL_D V& at(int e) { return a[e]; }
};

template <typename V>
struct SmemCol {
    V* base;     // &buf[t]
    int stride;  // elements between rows
    CHOL_D V& at(int e) { return base[e * stride]; }
};

// Registers hold the whole matrix when its packed triangle takes at most this
// many 32-bit words; larger matrices are worked in place in shared memory.
constexpr int kRegWords = 144;

template <typename V, int N>
constexpr bool lane_in_regs() { return tri(N) * traits<V>::words <= kRegWords; }

// Threads per CTA of the lane kernel: as many as fit in ~96 KB of staging.
template <typename V, int N>
constexpr int lane_threads() {
    constexpr int bytes = tri(N) * (int)sizeof(V);
    return bytes * 128 <= 98304 ? 128 : bytes * 64 <= 98304 ? 64 : 32;
}
template <typename V, int N>
constexpr int lane_stride() { return lane_threads<V, N>() + 1; }
template <typename V, int N>
constexpr size_t lane_smem_bytes() {
    return (size_t)tri(N) * lane_stride<V, N>() * sizeof(V) + (size_t)lane_threads<V, N>() * sizeof(int) +
           2 * (size_t)tri(N) * sizeof(uint8_t) + 16;
}

// ---------------------------------------------------------------------------
// Lane kernel: one matrix per thread.
// ---------------------------------------------------------------------------
template <typename V, int N>
__global__ void __launch_bounds__(lane_threads<V, N>())
k_lane(BatchParams p) {
    constexpr int THREADS = lane_threads<V, N>();
    constexpr int TN = tri(N);
    constexpr int LD = lane_stride<V, N>();
    using R = typename traits<V>::real;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* buf = reinterpret_cast<V*>(smem_raw);                                  // [TN][LD]
    int* s_info = reinterpret_cast<int*>(buf + (size_t)TN * LD);              // [THREADS]
    uint8_t* s_i = reinterpret_cast<uint8_t*>(s_info + THREADS);              // [TN] row of element e
    uint8_t* s_j = s_i + TN;                                                  // [TN] column of element e

    for (int e = threadIdx.x; e < TN; e += THREADS) {
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
    const int t = threadIdx.x;
    __syncthreads();

    for (int chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
        const int base = chunk * THREADS;
        const int m = min(THREADS, count - base);
        // ---- stage: global -> shared (consecutive threads read consecutive elements of a matrix)
        for (int f = t; f < m * TN; f += THREADS) {
            const int q = f / TN, e = f - q * TN;
            const int64_t b = member_index(p, N, base + q);
            const int64_t o = matrix_offset(p, N, b);
            const int64_t g = p.layout ? (int64_t)e : (int64_t)s_i[e] * N + s_j[e];
            buf[e * LD + q] = A[o + g];
        }
        __syncthreads();
        // ---- compute: thread t owns matrix base + t
        int info = 0;
        if (t < m) {
            R dinv[N];
            if constexpr (lane_in_regs<V, N>()) {
                RegMat<V, TN> r;
#pragma unroll
                for (int e = 0; e < TN; ++e) r.a[e] = buf[e * LD + t];
                info = factor_unrolled<V, N>(r, dinv);
                if (p.R && p.want_inv) {
                    // keep R for the store stage in the upper rows of the staging
                    // buffer?  No: R and X share storage, so R is stored here.
                    const int64_t b = member_index(p, N, base + t);
                    const int64_t o = matrix_offset(p, N, b);
#pragma unroll
                    for (int e = 0; e < TN; ++e) {
                        const int64_t g = p.layout ? (int64_t)e : (int64_t)s_i[e] * N + s_j[e];
                        Ro[o + g] = info ? nan_v<V>() : r.a[e];
                    }
                }
                if (p.want_inv) inverse_unrolled<V, N>(r, dinv);
#pragma unroll
                for (int e = 0; e < TN; ++e) buf[e * LD + t] = r.a[e];
            } else {
                SmemCol<V> s{buf + t, LD};
                info = factor_unrolled<V, N>(s, dinv);
                if (p.R && p.want_inv) {
                    const int64_t b = member_index(p, N, base + t);
                    const int64_t o = matrix_offset(p, N, b);
                    for (int e = 0; e < TN; ++e) {
                        const int64_t g = p.layout ? (int64_t)e : (int64_t)s_i[e] * N + s_j[e];
                        Ro[o + g] = info ? nan_v<V>() : buf[e * LD + t];
                    }
                }
                if (p.want_inv) inverse_unrolled<V, N>(s, dinv);
            }
            s_info[t] = info;
        }
        __syncthreads();
        // ---- store: shared -> global
        V* out = p.want_inv ? Xo : Ro;
        for (int f = t; f < m * TN; f += THREADS) {
            const int q = f / TN, e = f - q * TN;
            const int64_t b = member_index(p, N, base + q);
            const int64_t o = matrix_offset(p, N, b);
            const int i = s_i[e], j = s_j[e];
            const bool bad = s_info[q] != 0;
            V v = bad ? nan_v<V>() : buf[e * LD + q];
            if (p.layout) {
                out[o + e] = v;
            } else {
                out[o + (int64_t)i * N + j] = v;
                if (i != j) {
                    if (!p.want_inv) out[o + (int64_t)j * N + i] = bad ? nan_v<V>() : zero_v<V>();
                    else if (p.fill_lower) out[o + (int64_t)j * N + i] = conj_v(v);
                }
            }
        }
        if (!p.want_inv || p.R == nullptr) {
            // nothing else to write
        } else if (!p.layout) {
            // dense R: zero its strictly lower part
            for (int f = t; f < m * TN; f += THREADS) {
                const int q = f / TN, e = f - q * TN;
                const int i = s_i[e], j = s_j[e];
                if (i == j) continue;
                const int64_t b = member_index(p, N, base + q);
                const int64_t o = matrix_offset(p, N, b);
                Ro[o + (int64_t)j * N + i] = s_info[q] ? nan_v<V>() : zero_v<V>();
            }
        }
        if (p.info) {
            for (int q = t; q < m; q += THREADS) p.info[member_index(p, N, base + q)] = s_info[q];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Warp kernel: one matrix per warp, runtime order N (<= 64), lanes own the
// columns j = lane and j = lane + 32.  The matrix is a padded dense square
// in shared memory (row stride N+1).
// ---------------------------------------------------------------------------
template <typename V>
__global__ void k_warp(BatchParams p, int N, int warps_per_cta) {
    using R = typename traits<V>::real;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int LD = N + 1;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    V* S = reinterpret_cast<V*>(smem_raw) + (size_t)w * N * LD;
    const V* A = static_cast<const V*>(p.A);
    V* Xo = static_cast<V*>(p.X);
    V* Ro = static_cast<V*>(p.R);
    const int count = class_count(p, N);
    const int TN = tri(N);

    for (int k0 = blockIdx.x * warps_per_cta + w; k0 < count; k0 += gridDim.x * warps_per_cta) {
        const int64_t b = member_index(p, N, k0);
        const int64_t o = matrix_offset(p, N, b);
        // load the upper triangle
        if (p.layout) {
            for (int e = lane; e < TN; e += 32) {
                int i = 0;
                while (pidx(N, i + 1, i + 1) <= e && i + 1 < N) ++i;
                const int j = e - pidx(N, i, i) + i;
                S[i * LD + j] = A[o + e];
            }
        } else {
            for (int i = 0; i < N; ++i)
                for (int j = i + lane; j < N; j += 32) S[i * LD + j] = A[o + (int64_t)i * N + j];
        }
        __syncwarp();
        // ---- factor, Eqs. 3-4, row by row
        int info = 0;
        for (int i = 0; i < N; ++i) {
            V s0 = zero_v<V>(), s1 = zero_v<V>();
            const int j0 = lane, j1 = lane + 32;
            if (j0 >= i && j0 < N) {
                s0 = S[i * LD + j0];
                for (int k = 0; k < i; ++k) s0 = fnma_conj(S[k * LD + i], S[k * LD + j0], s0);
            }
            if (j1 >= i && j1 < N) {
                s1 = S[i * LD + j1];
                for (int k = 0; k < i; ++k) s1 = fnma_conj(S[k * LD + i], S[k * LD + j1], s1);
            }
            // pivot: column i lives in lane i & 31, slot i >> 5
            R tsrc = re_of((i < 32) ? s0 : s1);
            R tt = __shfl_sync(0xffffffffu, tsrc, i & 31);
            if (info == 0 && !pivot_ok(tt)) info = i + 1;
            const R rii = sqrt(tt);
            const R inv = R(1) / rii;
            if (j0 > i && j0 < N) S[i * LD + j0] = scale_v(s0, inv);
            if (j1 > i && j1 < N) S[i * LD + j1] = scale_v(s1, inv);
            if (lane == (i & 31)) S[i * LD + i] = from_real<V>(rii);
            __syncwarp();
        }
        if (p.R) {
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
        if (p.want_inv) {
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
                const R inv = R(1) / re_of(S[i * LD + i]);
                __syncwarp();
                R sd = R(0);
                if (j0 > i && j0 < N) { V x = scale_v(a0, -inv); S[i * LD + j0] = x; sd = fma_re_conjb(r0, x, sd); }
                if (j1 > i && j1 < N) { V x = scale_v(a1, -inv); S[i * LD + j1] = x; sd = fma_re_conjb(r1, x, sd); }
#pragma unroll
                for (int d = 16; d > 0; d >>= 1) sd += __shfl_xor_sync(0xffffffffu, sd, d);
                __syncwarp();
                if (lane == 0) S[i * LD + i] = from_real<V>((inv - sd) * inv);
                __syncwarp();
            }
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
}

// ---------------------------------------------------------------------------
// Size-class bucketing for batches with per-matrix orders.
// ws layout: counts[72] | starts[72] | cursor[72] | pad to 1024 B | perm[batch]
// ---------------------------------------------------------------------------
constexpr int kClasses = 72;

__global__ void k_bucket_hist(int32_t batch, const int32_t* __restrict__ n, int32_t max_n, int32_t* counts,
                              int32_t* info, int* err);
__global__ void k_bucket_scan(int32_t* counts, int32_t* starts, int32_t* cursor);
__global__ void k_bucket_scatter(int32_t batch, const int32_t* __restrict__ n, int32_t max_n, int32_t* cursor,
                                 int32_t* perm);

}  // namespace cholinv
