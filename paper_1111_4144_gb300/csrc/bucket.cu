// Size-class bucketing of a batch with per-matrix orders: a histogram of
// n[b] whose last CTA takes the exclusive scan over the classes, then a
// scatter of the matrix indices into class order.  Every kernel is a plain
// grid-stride loop; no CTA waits on another, so nothing here can stall.
#include "batched.cuh"

namespace cholinv {

__global__ void k_bucket_hist(int32_t batch, const int32_t* __restrict__ n, int32_t max_n, uint64_t m0, uint64_t m1,
                              int32_t* counts, int32_t* starts, int32_t* cursor, unsigned* done, int32_t* info,
                              int* err) {
    __shared__ int sh[kClasses];
    for (int c = threadIdx.x; c < kClasses; c += blockDim.x) sh[c] = 0;
    __syncthreads();
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < batch; b += (int64_t)gridDim.x * blockDim.x) {
        const int nb = n[b];
        if (nb < 0 || nb > max_n || (nb > 0 && !order_allowed(m0, m1, nb))) {
            if (info) info[b] = -1;
            report_error(err, CHOL_ERR_ARG);
        } else if (nb == 0) {
            if (info) info[b] = 0;
        } else {
            atomicAdd(&sh[nb], 1);
        }
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
        int nb = 0, rank = 0;
        if (b < batch) {
            nb = n[b];
            if (nb > 0 && nb <= max_n && order_allowed(m0, m1, nb)) rank = atomicAdd(&cnt[nb], 1);
            else nb = 0;
        }
        __syncthreads();
        for (int c = threadIdx.x; c < kClasses; c += blockDim.x)
            if (cnt[c]) basec[c] = atomicAdd(&cursor[c], cnt[c]);
        __syncthreads();
        if (nb > 0) perm[basec[nb] + rank] = (int32_t)b;
        __syncthreads();
    }
}

}  // namespace cholinv
