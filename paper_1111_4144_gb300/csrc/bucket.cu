// Size-class bucketing of a batch with per-matrix orders: a histogram of
// n[b] whose last CTA takes the exclusive scan over the classes, then a
// scatter of the matrix indices into class order.  Every kernel is a plain
// grid-stride loop; no CTA waits on another, so nothing here can stall.
#include "batched.cuh"

namespace cholinv {

// One shared-memory atomic per distinct class among a warp's lanes (the
// lanes of a class elect a leader): a batch of few orders would otherwise
// serialise 32 atomics per warp on the same counter.  Returns, for a lane
// of class c >= 0, its rank among the lanes of c, with *base the value the
// counter held before the warp's lanes of c were added.
CHOL_D int warp_aggregated_add(int* counter_of_c, int c, int& base) {
    const unsigned active = __activemask();
    const unsigned peers = __match_any_sync(active, c);
    const int leader = __ffs(peers) - 1;
    const int lane = threadIdx.x & 31;
    int b = 0;
    if (lane == leader && c >= 0) b = atomicAdd(counter_of_c, __popc(peers));
    base = __shfl_sync(active, b, leader);
    return __popc(peers & ((1u << lane) - 1u));
}

__global__ void k_bucket_hist(int32_t batch, const int32_t* __restrict__ n, int32_t max_n, uint64_t m0, uint64_t m1,
                              int32_t* counts, int32_t* starts, int32_t* cursor, unsigned* done, int32_t* info,
                              int* err) {
    __shared__ int sh[kClasses];
    for (int c = threadIdx.x; c < kClasses; c += blockDim.x) sh[c] = 0;
    __syncthreads();
    // every lane of a warp runs the same number of rounds, so the warp-wide
    // match below always sees the whole warp
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t b0 = (int64_t)blockIdx.x * blockDim.x; b0 < batch; b0 += stride) {
        const int64_t b = b0 + threadIdx.x;
        int cls = -1;  // -1: no class (outside the batch, empty or invalid)
        if (b < batch) {
            const int nb = n[b];
            if (nb < 0 || nb > max_n || (nb > 0 && !order_allowed(m0, m1, nb))) {
                if (info) info[b] = -1;
                report_error(err, CHOL_ERR_ARG);
            } else if (nb == 0) {
                if (info) info[b] = 0;
            } else {
                cls = nb;
            }
        }
        int base;
        warp_aggregated_add(&sh[cls < 0 ? 0 : cls], cls, base);
    }
    __syncthreads();
    for (int c = threadIdx.x; c < kClasses; c += blockDim.x)
        if (sh[c]) atomicAdd(&counts[c], sh[c]);
    // the last CTA to finish turns the counts into class starts (no CTA waits:
    // each one only adds to a counter after its own counts are visible)
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        int s = 0;
        for (int c = 0; c < kClasses; ++c) {
            const int v = *reinterpret_cast<volatile int32_t*>(&counts[c]);
            starts[c] = s;
            cursor[c] = s;
            s += v;
        }
        *done = 0u;  // ready for the next call (the counters are cleared before each call too)
    }
}

__global__ void k_bucket_scatter(int32_t batch, const int32_t* __restrict__ n, int32_t max_n, uint64_t m0,
                                 uint64_t m1, int32_t* cursor, int32_t* perm) {
    __shared__ int cnt[kClasses];
    __shared__ int basec[kClasses];
    for (int64_t tile = blockIdx.x; tile * blockDim.x < batch; tile += gridDim.x) {
        for (int c = threadIdx.x; c < kClasses; c += blockDim.x) cnt[c] = 0;
        __syncthreads();
        const int64_t b = tile * blockDim.x + threadIdx.x;
        int nb = 0;
        if (b < batch) {
            nb = n[b];
            if (!(nb > 0 && nb <= max_n && order_allowed(m0, m1, nb))) nb = 0;
        }
        int base;
        const int within = warp_aggregated_add(&cnt[nb > 0 ? nb : 0], nb > 0 ? nb : -1, base);
        const int rank = base + within;
        __syncthreads();
        for (int c = threadIdx.x; c < kClasses; c += blockDim.x)
            if (cnt[c]) basec[c] = atomicAdd(&cursor[c], cnt[c]);
        __syncthreads();
        if (nb > 0) perm[basec[nb] + rank] = (int32_t)b;
        __syncthreads();
    }
}

}  // namespace cholinv
