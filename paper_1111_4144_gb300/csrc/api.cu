// C-ABI of the cholinv library (declared in include/cholinv.h): host-side
// argument validation, size-class bucketing, kernel dispatch, plans (CUDA
// graphs) and the device error word.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "batched.cuh"
#include "blocked.h"
#include "dispatch.h"

// The per-device error word; kernels receive its address as an argument.
__device__ int g_chol_error_word;
// Matrices redone with FP64 pivots under CHOL_FLAG_PIVOT64_AUTO (per device).
__device__ unsigned long long g_chol_redo_count;
// Work counter of a single-launch call on a uniform batch (per device).
__device__ int g_chol_single_work;

namespace cholinv {

namespace {

constexpr int kMaxDevices = 64;
constexpr int kBatchedMaxN = 64;

struct DevState {
    bool init = false;
    int sms = 0;
    int* err = nullptr;
    unsigned long long* redo = nullptr;
    int* work = nullptr;  // single-launch work counter of uniform batches
};
DevState g_dev[kMaxDevices];
std::mutex g_dev_mu;

cudaError_t dev_state(DevState** out) {
    int d = 0;
    cudaError_t e = cudaGetDevice(&d);
    if (e != cudaSuccess) return e;
    if (d < 0 || d >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_dev_mu);
    DevState& s = g_dev[d];
    if (!s.init) {
        e = cudaDeviceGetAttribute(&s.sms, cudaDevAttrMultiProcessorCount, d);
        if (e != cudaSuccess) return e;
        e = cudaGetSymbolAddress(reinterpret_cast<void**>(&s.err), g_chol_error_word);
        if (e != cudaSuccess) return e;
        e = cudaGetSymbolAddress(reinterpret_cast<void**>(&s.redo), g_chol_redo_count);
        if (e != cudaSuccess) return e;
        e = cudaGetSymbolAddress(reinterpret_cast<void**>(&s.work), g_chol_single_work);
        if (e != cudaSuccess) return e;
        s.init = true;
    }
    *out = &s;
    return cudaSuccess;
}

// counts | starts | cursor (kClasses int32 each) | done | single-launch work counter, padded
constexpr size_t kWsHeader = 1024;
constexpr int kWsHeaderInts = 3 * kClasses + 2;
static_assert(kWsHeaderInts * sizeof(int32_t) <= kWsHeader, "bucketing header overlaps the permutation");

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

size_t ws_need_batched(int32_t batch, int32_t has_sizes) {
    if (!has_sizes || batch <= 0) return 0;
    return kWsHeader + align_up((size_t)batch * sizeof(int32_t), 256);
}

chol_opts_t opts_or_default(const chol_opts_t* o) {
    chol_opts_t d;
    d.prec = CHOL_PREC_NATIVE;
    d.refine_steps = 0;
    d.fill_lower = 0;
    d.layout = 0;
    d.flags = 0;
    d.reserved = 0;
    d.orders = 0;
    return o ? *o : d;
}

bool is_fp32(chol_dtype_t dt) { return dt == CHOL_F32 || dt == CHOL_C64; }

chol_status_t check_common(chol_dtype_t dt, int32_t batch, int32_t max_n, const chol_opts_t& o) {
    if (dt < CHOL_F32 || dt > CHOL_C128) return CHOL_ERR_ARG;
    if (batch < 0) return CHOL_ERR_ARG;
    if (max_n < 1) return CHOL_ERR_ARG;
    if (o.layout != 0 && o.layout != 1) return CHOL_ERR_ARG;
    if (o.reserved != 0) return CHOL_ERR_ARG;
    if (o.prec < CHOL_PREC_NATIVE || o.prec > CHOL_PREC_BF16_REFINE) return CHOL_ERR_ARG;
    if (o.refine_steps < -1 || o.refine_steps > 2) return CHOL_ERR_ARG;
    if (o.flags & ~(CHOL_FLAG_PIVOT64 | CHOL_FLAG_GRAD_UPPER | CHOL_FLAG_LDL | CHOL_FLAG_PIVOT64_AUTO |
                    CHOL_FLAG_RESIDUAL_FP64 | CHOL_FLAG_METHOD_ES | CHOL_FLAG_METHOD_TMO | CHOL_FLAG_SINGLE_LAUNCH))
        return CHOL_ERR_ARG;
    if ((o.flags & CHOL_FLAG_LDL) && (o.flags & (CHOL_FLAG_PIVOT64 | CHOL_FLAG_PIVOT64_AUTO)))
        return CHOL_ERR_UNSUPPORTED;
    if ((o.flags & CHOL_FLAG_METHOD_ES) && (o.flags & CHOL_FLAG_METHOD_TMO)) return CHOL_ERR_ARG;
    if ((o.flags & (CHOL_FLAG_METHOD_ES | CHOL_FLAG_METHOD_TMO)) && (o.flags & CHOL_FLAG_LDL))
        return CHOL_ERR_UNSUPPORTED;
    if (max_n > kBatchedMaxN) return CHOL_ERR_UNSUPPORTED;
    if (o.prec == CHOL_PREC_TF32_REFINE || o.prec == CHOL_PREC_BF16_REFINE) return CHOL_ERR_UNSUPPORTED;
    if (o.prec == CHOL_PREC_FP32_REFINE && !is_fp32(dt)) return CHOL_ERR_UNSUPPORTED;
    return CHOL_OK;
}

chol_status_t check_ws(int32_t batch, const int32_t* n, void* ws, size_t ws_bytes) {
    const size_t need = ws_need_batched(batch, n != nullptr);
    if (need == 0) return CHOL_OK;
    if (ws == nullptr || ws_bytes < need) return CHOL_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return CHOL_ERR_WORKSPACE;
    return CHOL_OK;
}

cudaError_t launch_dtype_class(chol_dtype_t dt, const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry) {
    switch (dt) {
        case CHOL_F32: return launch_class_f32(p, cls, upper, s, dry);
        case CHOL_F64: return launch_class_f64(p, cls, upper, s, dry);
        case CHOL_C64: return launch_class_c64(p, cls, upper, s, dry);
        case CHOL_C128: return launch_class_c128(p, cls, upper, s, dry);
    }
    return cudaErrorInvalidValue;
}

// Timing events of a plan being captured (CHOL_FLAG_PLAN_TIMING): recorded
// around each size-class kernel on the stream that runs it.
struct ClassTiming {
    cudaEvent_t start[kClasses];
    cudaEvent_t end[kClasses];
    bool used[kClasses];
};
thread_local ClassTiming* t_timing = nullptr;

cudaError_t launch_class_timed(chol_dtype_t dt, const BatchParams& p, int c, cudaStream_t st) {
    cudaError_t e;
    // cudaEventRecordExternal: inside a capture this makes a real event-record
    // node (a plain record would only express a dependency)
    if (t_timing && (e = cudaEventRecordWithFlags(t_timing->start[c], st, cudaEventRecordExternal)) != cudaSuccess)
        return e;
    if ((e = launch_dtype_class(dt, p, c, p.batch, st, false)) != cudaSuccess) return e;
    if (t_timing) {
        if ((e = cudaEventRecordWithFlags(t_timing->end[c], st, cudaEventRecordExternal)) != cudaSuccess) return e;
        t_timing->used[c] = true;
    }
    return cudaSuccess;
}

// Side streams on which the class kernels of one call run side by side (per
// host thread and device; created outside any stream capture, kept for the
// life of the thread).  A batch of many orders with a few thousand matrices
// each (orders 2..64, 262,144 matrices) leaves most of the GPU idle when its
// class kernels run one after another: each fills a fraction of the SMs and
// the step costs the sum of their latencies.
constexpr int kForkStreams = 8;
constexpr int kForkMinClasses = 8;
struct ClassFork {
    bool ok = false;
    cudaStream_t side[kForkStreams];
    cudaEvent_t fork;
    cudaEvent_t join[kForkStreams];
};
thread_local ClassFork t_fork[kMaxDevices];

// The calling thread's side streams for the current device, created if
// `may_create`; nullptr if they do not exist (or cannot be made).
ClassFork* class_fork(bool may_create) {
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDevices) return nullptr;
    ClassFork& f = t_fork[d];
    if (f.ok || !may_create) return f.ok ? &f : nullptr;
    bool good = cudaEventCreateWithFlags(&f.fork, cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; good && k < kForkStreams; ++k)
        good = cudaStreamCreateWithFlags(&f.side[k], cudaStreamNonBlocking) == cudaSuccess &&
               cudaEventCreateWithFlags(&f.join[k], cudaEventDisableTiming) == cudaSuccess;
    if (!good) {
        cudaGetLastError();
        return nullptr;
    }
    f.ok = true;
    return &f;
}

// Every size class of a batch, largest orders first: one class for uniform
// batches, otherwise every class 1..max_n (a class kernel with no members
// exits at once).  `present` (optional, host memory): present[c] != 0 for
// the orders that occur in the batch, when the caller knows them; other
// classes are skipped.
// With kForkMinClasses or more classes the kernels are dealt round-robin to
// side streams forked from `s` and joined back (inside a capture: parallel
// branches of the graph).  Fewer, larger classes each fill the GPU and run on
// `s` in order (three classes of 349,525 matrices measured no faster side by
// side), and so do plans with per-kernel timing, whose events must bracket
// one kernel at a time.
cudaError_t launch_dtype(chol_dtype_t dt, const BatchParams& p, cudaStream_t s, bool dry,
                         const uint8_t* present = nullptr) {
    if (p.cls_count == nullptr) {
        if (dry) return launch_dtype_class(dt, p, p.max_n, p.batch, s, true);
        return launch_class_timed(dt, p, p.max_n, s);
    }
    int nclasses = 0;
    for (int c = p.max_n; c >= 1; --c) nclasses += (!present || present[c]) ? 1 : 0;
    const bool want_fork = nclasses >= kForkMinClasses && t_timing == nullptr;
    if (dry || !want_fork) {
        // the dry pass (before a plan's capture) makes the side streams
        if (dry && want_fork) class_fork(true);
        for (int c = p.max_n; c >= 1; --c) {
            if (present && !present[c]) continue;
            cudaError_t e = dry ? launch_dtype_class(dt, p, c, p.batch, s, true) : launch_class_timed(dt, p, c, s);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return cudaGetLastError();
    ClassFork* f = class_fork(cap == cudaStreamCaptureStatusNone);
    if (f == nullptr) {
        for (int c = p.max_n; c >= 1; --c) {
            if (present && !present[c]) continue;
            cudaError_t e = launch_class_timed(dt, p, c, s);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    const int used = std::min(nclasses, kForkStreams);
    cudaError_t e = cudaEventRecord(f->fork, s);
    for (int k = 0; e == cudaSuccess && k < used; ++k) e = cudaStreamWaitEvent(f->side[k], f->fork, 0);
    int next = 0;
    for (int c = p.max_n; e == cudaSuccess && c >= 1; --c) {
        if (present && !present[c]) continue;
        e = launch_class_timed(dt, p, c, f->side[next]);
        next = (next + 1) % used;
    }
    // join every side stream that waited on the fork, also after an error,
    // so that a capture in progress is left with no unjoined work
    for (int k = 0; k < used; ++k) {
        cudaError_t j = cudaEventRecord(f->join[k], f->side[k]);
        if (j == cudaSuccess) j = cudaStreamWaitEvent(s, f->join[k], 0);
        if (e == cudaSuccess) e = j;
    }
    return e;
}

// Enqueue bucketing (if per-matrix sizes) and every class kernel.
chol_status_t enqueue_batched(chol_dtype_t dt, BatchParams p, void* ws, cudaStream_t s, bool dry,
                              const uint8_t* present = nullptr) {
    // a caller-stated order set: kernels for those orders only
    uint8_t from_mask[kClasses];
    if (present == nullptr && p.n != nullptr && (~p.order_mask[0] | ~p.order_mask[1]) != 0) {
        for (int c = 0; c < kClasses; ++c)
            from_mask[c] = c >= 1 && c <= p.max_n && order_allowed(p.order_mask[0], p.order_mask[1], c);
        present = from_mask;
    }
    DevState* ds = nullptr;
    if (dev_state(&ds) != cudaSuccess) return CHOL_ERR_CUDA;
    p.err = ds->err;
    p.redo_count = ds->redo;
    if (p.n != nullptr) {
        char* w = static_cast<char*>(ws);
        int32_t* counts = reinterpret_cast<int32_t*>(w);
        int32_t* starts = counts + kClasses;
        int32_t* cursor = starts + kClasses;
        int32_t* perm = reinterpret_cast<int32_t*>(w + kWsHeader);
        p.cls_count = counts;
        p.cls_start = starts;
        p.perm = perm;
        if (!dry) {
            // counts and the done counter (right after cursor) cleared together
            unsigned* done = reinterpret_cast<unsigned*>(cursor + kClasses);
            if (cudaMemsetAsync(counts, 0, kWsHeaderInts * sizeof(int32_t), s) != cudaSuccess)
                return CHOL_ERR_CUDA;
            const int threads = 256;
            const int grid = (int)std::min<int64_t>(((int64_t)p.batch + threads - 1) / threads, (int64_t)ds->sms * 8);
            k_bucket_hist<<<grid, threads, 0, s>>>(p.batch, p.n, p.max_n, p.order_mask[0], p.order_mask[1], counts,
                                                   starts, cursor, done, p.info, p.err);
            k_bucket_scatter<<<grid, threads, 0, s>>>(p.batch, p.n, p.max_n, p.order_mask[0], p.order_mask[1], cursor,
                                                      perm);
            if (cudaGetLastError() != cudaSuccess) return CHOL_ERR_CUDA;
        }
    }
    if (p.flags & CHOL_FLAG_SINGLE_LAUNCH) {
        // one persistent launch over every order (its work counter follows the header's done word)
        int* work = p.n != nullptr ? reinterpret_cast<int32_t*>(ws) + 3 * kClasses + 1 : nullptr;
        if (work == nullptr) {
            // uniform batch: no bucketing workspace; the counter lives in the device state
            work = ds->work;
            if (!dry && cudaMemsetAsync(work, 0, sizeof(int), s) != cudaSuccess) return CHOL_ERR_CUDA;
        }
        if (launch_single(dt, p, work, s, dry) != cudaSuccess) return CHOL_ERR_CUDA;
    } else if (launch_dtype(dt, p, s, dry, present) != cudaSuccess) {
        return CHOL_ERR_CUDA;
    }
    // matrices whose FP32 pivots cancelled, again with FP64 pivots
    if ((p.flags & CHOL_FLAG_PIVOT64_AUTO) && !(p.flags & CHOL_FLAG_PIVOT64) && is_fp32(dt) &&
        launch_redo(dt, p, s, dry) != cudaSuccess)
        return CHOL_ERR_CUDA;
    return CHOL_OK;
}

chol_status_t inv_validate(chol_dtype_t dt, int32_t batch, const int32_t* n, int32_t max_n, const void* A,
                           void* X, const int32_t* info, const chol_opts_t& o, void* ws, size_t ws_bytes) {
    chol_status_t st = check_common(dt, batch, max_n, o);
    if (st != CHOL_OK) return st;
    if (batch == 0) return CHOL_OK;
    if (A == nullptr || X == nullptr) return CHOL_ERR_ARG;
    if ((o.flags & CHOL_FLAG_PIVOT64_AUTO) && info == nullptr) return CHOL_ERR_ARG;  // the redo list lives in info
    if (o.prec == CHOL_PREC_FP32_REFINE && o.refine_steps != 0 && X == A) return CHOL_ERR_ARG;
    return check_ws(batch, n, ws, ws_bytes);
}

// The inverse with its optional refinement pass.
chol_status_t enqueue_inv(chol_dtype_t dt, BatchParams p, void* ws, cudaStream_t s, bool dry, const chol_opts_t& o,
                          const uint8_t* present = nullptr) {
    chol_status_t st = enqueue_batched(dt, p, ws, s, dry, present);
    if (st != CHOL_OK) return st;
    if (o.prec == CHOL_PREC_FP32_REFINE && o.refine_steps != 0) {
        BatchParams q = p;
        DevState* ds = nullptr;
        if (dev_state(&ds) != cudaSuccess) return CHOL_ERR_CUDA;
        q.err = ds->err;
        const int steps = o.refine_steps > 0 ? o.refine_steps : 1;
        if (launch_refine(dt, q, steps, o.refine_steps < 0, s, dry) != cudaSuccess) return CHOL_ERR_CUDA;
    }
    return CHOL_OK;
}

BatchParams make_params(int32_t batch, const int32_t* n, const int64_t* off, int32_t max_n, const void* A,
                        void* R, void* X, int32_t* info, const chol_opts_t& o, int want_inv) {
    BatchParams p;
    std::memset(&p, 0, sizeof(p));
    p.batch = batch;
    p.n = n;
    p.off = off;
    p.max_n = max_n;
    p.layout = o.layout;
    p.fill_lower = o.layout == 0 ? o.fill_lower : 0;
    p.want_inv = want_inv;
    p.A = A;
    p.R = R;
    p.X = X;
    p.info = info;
    p.flags = o.flags;
    // the caller's order set (bit c-1 of o.orders for order c) as bit c of the mask
    p.order_mask[0] = p.order_mask[1] = ~0ull;
    if (n != nullptr && o.orders != 0) {
        p.order_mask[0] = o.orders << 1;
        p.order_mask[1] = o.orders >> 63;
    }
    p.aligned16 = ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(R) | reinterpret_cast<uintptr_t>(X)) %
                   16) == 0;
    return p;
}

// Orders above kBatchedMaxN take the blocked path: uniform batches of dense
// real matrices (FP32, FP64), processed one matrix at a time.
chol_status_t blocked_validate(chol_dtype_t dt, int32_t batch, const int32_t* n, const int64_t* off, int32_t max_n,
                               const chol_opts_t& o, size_t need, void* ws, size_t ws_bytes) {
    if (dt < CHOL_F32 || dt > CHOL_C128 || batch < 0) return CHOL_ERR_ARG;
    if (o.layout != 0 && o.layout != 1) return CHOL_ERR_ARG;
    if (o.reserved != 0) return CHOL_ERR_ARG;
    if (o.prec < CHOL_PREC_NATIVE || o.prec > CHOL_PREC_BF16_REFINE) return CHOL_ERR_ARG;
    if (o.refine_steps < -1 || o.refine_steps > 2) return CHOL_ERR_ARG;
    if (o.flags & CHOL_FLAG_LDL) return CHOL_ERR_UNSUPPORTED;
    if (o.flags & ~(CHOL_FLAG_PIVOT64 | CHOL_FLAG_GRAD_UPPER | CHOL_FLAG_TF32_SINGLE | CHOL_FLAG_PIVOT64_AUTO |
                    CHOL_FLAG_RESIDUAL_FP64))
        return CHOL_ERR_ARG;
    if (n != nullptr || off != nullptr || o.layout != 0) return CHOL_ERR_UNSUPPORTED;
    if (o.prec == CHOL_PREC_BF16_REFINE) return CHOL_ERR_UNSUPPORTED;
    if ((o.prec == CHOL_PREC_FP32_REFINE || o.prec == CHOL_PREC_TF32_REFINE) && !is_fp32(dt))
        return CHOL_ERR_UNSUPPORTED;
    // complex matrices run as their real embedding of order 2 max_n
    const bool cplx = dt == CHOL_C64 || dt == CHOL_C128;
    if ((cplx ? 2 * (int64_t)max_n : (int64_t)max_n) > 1 << 16) return CHOL_ERR_UNSUPPORTED;
    if (batch > 0 && (ws == nullptr || ws_bytes < need || reinterpret_cast<uintptr_t>(ws) % 256 != 0))
        return CHOL_ERR_WORKSPACE;
    return CHOL_OK;
}

// Bytes of one packed matrix array (A or X) of an MMSE call in the workspace.
size_t mmse_ws_matrices(chol_dtype_t dt, int32_t batch, int32_t max_n) {
    const size_t es = dt == CHOL_F32 ? 4 : dt == CHOL_C128 ? 16 : 8;
    return align_up((size_t)batch * tri(max_n) * es, 256);
}

// ---------------------------------------------------------------------------
// Host-resident batches (chol_inv_batched_host): chunks of whole matrices
// move through kHostSlots device slots on four internal streams (copy in,
// two for the kernels of alternate chunks, copy out).
// ---------------------------------------------------------------------------
constexpr int kHostSlots = 4;
constexpr int kHostChunks = 16;         // chunks per call (fewer for small batches)
constexpr int kHostMinChunk = 8192;     // matrices
// Copies between pinned host memory and the device run at the link's rate
// only from host addresses on 128-byte boundaries (measured on GB300: a
// 16-byte aligned start cuts the copy-in rate from 208 to 176 GB/s, and
// both directions together from 314 to 226 GB/s).  Each chunk's copies start
// on such a boundary, with the chunk placed at the same offset in its slot.
constexpr size_t kHostAlign = 128;

int64_t host_chunk_matrices(int32_t batch) {
    const int64_t c = ((int64_t)batch + kHostChunks - 1) / kHostChunks;
    return std::max<int64_t>(std::min<int64_t>(c, batch), std::min<int64_t>(kHostMinChunk, batch));
}
size_t elem_size(chol_dtype_t dt) { return dt == CHOL_F32 ? 4 : dt == CHOL_C128 ? 16 : 8; }
int64_t matrix_elems(int layout, int64_t n) { return layout ? n * (n + 1) / 2 : n * n; }

// The workspace of the host path: the whole batch's orders, offsets and
// info (each copied in one piece: per-chunk copies of a few hundred KB cost
// more in copy-engine and event latency than in bytes), then kHostSlots
// slots of A, X and the bucketing workspace for one chunk.
struct HostSlotLayout {
    size_t n, off, info;     // byte offsets of the whole-batch arrays
    size_t slots;            // byte offset of the first slot
    size_t a, x, ws, total;  // byte offsets within one slot, and its size
    size_t bytes;            // the whole workspace
};
HostSlotLayout host_slot_layout(chol_dtype_t dt, int32_t batch, int32_t max_n, int layout, bool has_sizes) {
    const int64_t mc = host_chunk_matrices(batch);
    // room for a chunk placed up to kHostAlign - 1 bytes into its slot
    const size_t data = align_up((size_t)mc * matrix_elems(layout, max_n) * elem_size(dt) + kHostAlign, 256);
    HostSlotLayout l;
    l.n = 0;
    l.off = l.n + (has_sizes ? align_up((size_t)batch * sizeof(int32_t), 256) : 0);
    l.info = l.off + (has_sizes ? align_up((size_t)batch * sizeof(int64_t), 256) : 0);
    l.slots = l.info + align_up((size_t)batch * sizeof(int32_t), 256);
    l.a = 0;
    l.x = l.a + data;
    l.ws = l.x + data;
    l.total = l.ws + ws_need_batched((int32_t)mc, has_sizes);
    l.bytes = l.slots + l.total * kHostSlots;
    return l;
}

// Per-device streams of the host path: one per pipeline stage (copy in,
// kernels, copy out), the events that chain a chunk through the stages and
// free its slot again, and those that fork the stages from and join them to
// the caller's stream.  Enqueueing holds the mutex.
struct HostStreams {
    cudaStream_t in = nullptr, run[2] = {}, out = nullptr;  // chunks alternate between the two kernel streams
    cudaEvent_t fork = nullptr, join[4] = {};
    cudaEvent_t loaded[kHostChunks] = {}, computed[kHostChunks] = {}, freed[kHostSlots] = {};
    std::mutex mu;
};
HostStreams* host_streams() {
    static std::mutex init_mu;
    static HostStreams* per_dev[kMaxDevices] = {};
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lk(init_mu);
    if (!per_dev[d]) {
        HostStreams* h = new HostStreams();
        auto ev = [](cudaEvent_t* e) { return cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess; };
        bool ok = cudaStreamCreateWithFlags(&h->in, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&h->run[0], cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&h->run[1], cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&h->out, cudaStreamNonBlocking) == cudaSuccess && ev(&h->fork);
        for (int k = 0; k < 4 && ok; ++k) ok = ev(&h->join[k]);
        for (int k = 0; k < kHostChunks && ok; ++k) ok = ev(&h->loaded[k]) && ev(&h->computed[k]);
        for (int k = 0; k < kHostSlots && ok; ++k) ok = ev(&h->freed[k]);
        if (!ok) {
            delete h;
            return nullptr;
        }
        per_dev[d] = h;
    }
    return per_dev[d];
}

int blocked_refine_steps(const chol_opts_t& o) {
    if (o.prec != CHOL_PREC_FP32_REFINE && o.prec != CHOL_PREC_TF32_REFINE) return 0;
    return o.refine_steps < 0 ? 1 : o.refine_steps;
}

// The blocked path has one matrix per call: CHOL_FLAG_PIVOT64_AUTO there
// means FP64 pivots for its diagonal blocks.
int blocked_pivot64(const chol_opts_t& o) { return (o.flags & (CHOL_FLAG_PIVOT64 | CHOL_FLAG_PIVOT64_AUTO)) ? 1 : 0; }

// Tensor-core mode of the blocked products (see blocked_run).
int blocked_tc(const chol_opts_t& o) {
    if (o.prec != CHOL_PREC_TF32_REFINE) return 0;
    return (o.flags & CHOL_FLAG_TF32_SINGLE) ? 1 : 2;
}

int* device_error_word() {
    DevState* ds = nullptr;
    return dev_state(&ds) == cudaSuccess ? ds->err : nullptr;
}

}  // namespace

DeviceInfo device_info() {
    DeviceInfo d;
    DevState* ds = nullptr;
    if (dev_state(&ds) == cudaSuccess) d.sms = ds->sms;
    if (d.sms <= 0) d.sms = 1;
    return d;
}

}  // namespace cholinv

using namespace cholinv;

struct chol_plan {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    ClassTiming* timing = nullptr;
};

extern "C" {

chol_status_t chol_factor_batched(chol_dtype_t dt, int32_t batch, const int32_t* n, const int64_t* off,
                                  int32_t max_n, const void* A, void* R, int32_t* info,
                                  const chol_opts_t* opts, void* ws, size_t ws_bytes, void* stream) {
    const chol_opts_t o = opts_or_default(opts);
    if (max_n > kBatchedMaxN) {
        chol_status_t sb = blocked_validate(dt, batch, n, off, max_n, o,
                                            blocked_workspace_bytes(dt, max_n, 0), ws, ws_bytes);
        if (sb != CHOL_OK || batch == 0) return sb;
        if (A == nullptr || R == nullptr) return CHOL_ERR_ARG;
        if (dt == CHOL_C64 || dt == CHOL_C128) return CHOL_ERR_UNSUPPORTED;  // no complex R above order 64
        // the factor is formed in R itself (R is the working storage)
        return blocked_run(dt, batch, max_n, A, nullptr, R, info, blocked_pivot64(o), 0, 0, 0, blocked_tc(o),
                           device_error_word(), ws, static_cast<cudaStream_t>(stream));
    }
    chol_status_t st = check_common(dt, batch, max_n, o);
    if (st != CHOL_OK) return st;
    if (batch == 0) return CHOL_OK;
    if (A == nullptr || R == nullptr) return CHOL_ERR_ARG;
    if ((o.flags & CHOL_FLAG_PIVOT64_AUTO) && info == nullptr) return CHOL_ERR_ARG;
    st = check_ws(batch, n, ws, ws_bytes);
    if (st != CHOL_OK) return st;
    BatchParams p = make_params(batch, n, off, max_n, A, R, nullptr, info, o, 0);
    return enqueue_batched(dt, p, ws, static_cast<cudaStream_t>(stream), false);
}

chol_status_t chol_inv_batched(chol_dtype_t dt, int32_t batch, const int32_t* n, const int64_t* off,
                               int32_t max_n, const void* A, void* R, void* X, int32_t* info,
                               const chol_opts_t* opts, void* ws, size_t ws_bytes, void* stream) {
    const chol_opts_t o = opts_or_default(opts);
    if (max_n > kBatchedMaxN) {
        const int rs = blocked_refine_steps(o);
        chol_status_t sb = blocked_validate(dt, batch, n, off, max_n, o, blocked_workspace_bytes(dt, max_n, rs), ws,
                                            ws_bytes);
        if (sb != CHOL_OK || batch == 0) return sb;
        if (A == nullptr || X == nullptr) return CHOL_ERR_ARG;
        if (X == A || (R != nullptr && (R == A || R == X))) return CHOL_ERR_ARG;
        if ((dt == CHOL_C64 || dt == CHOL_C128) && R != nullptr) return CHOL_ERR_UNSUPPORTED;
        return blocked_run(dt, batch, max_n, A, R, X, info, blocked_pivot64(o), rs,
                           (o.flags & CHOL_FLAG_RESIDUAL_FP64) ? 1 : 0, 1, blocked_tc(o),
                           device_error_word(), ws, static_cast<cudaStream_t>(stream));
    }
    chol_status_t st = inv_validate(dt, batch, n, max_n, A, X, info, o, ws, ws_bytes);
    if (st != CHOL_OK || batch == 0) return st;
    BatchParams p = make_params(batch, n, off, max_n, A, (R == X) ? nullptr : R, X, info, o, 1);
    return enqueue_inv(dt, p, ws, static_cast<cudaStream_t>(stream), false, o);
}

chol_status_t chol_inv_backward(chol_dtype_t dt, int32_t batch, const int32_t* n, const int64_t* off,
                                const int64_t* xoff, int32_t max_n, const void* X, const void* G, void* dA,
                                const chol_opts_t* opts, void* ws, size_t ws_bytes, void* stream) {
    (void)ws; (void)ws_bytes;
    const chol_opts_t o = opts_or_default(opts);
    chol_status_t st = check_common(dt, batch, max_n, o);
    if (st != CHOL_OK || batch == 0) return st;
    if (X == nullptr || G == nullptr || dA == nullptr) return CHOL_ERR_ARG;
    if (dA == X || dA == G) return CHOL_ERR_ARG;
    BwdParams p;
    std::memset(&p, 0, sizeof(p));
    p.batch = batch;
    p.n = n;
    p.off = off;
    p.xoff = xoff;
    p.max_n = max_n;
    p.layout = o.layout;
    p.X = X;
    p.G = G;
    p.dA = dA;
    p.flags = o.flags;
    if (launch_backward(dt, p, static_cast<cudaStream_t>(stream), false) != cudaSuccess) return CHOL_ERR_CUDA;
    return CHOL_OK;
}

chol_status_t chol_inv_batched_host(chol_dtype_t dt, int32_t batch, const int32_t* n_host, const int64_t* off_host,
                                    int32_t max_n, const void* A_host, void* X_host, int32_t* info_host,
                                    const chol_opts_t* opts, void* ws, size_t ws_bytes, void* stream) {
    chol_opts_t o = opts_or_default(opts);
    chol_status_t st = check_common(dt, batch, max_n, o);
    if (st != CHOL_OK) return st;
    if (max_n > kBatchedMaxN) return CHOL_ERR_UNSUPPORTED;
    if ((n_host == nullptr) != (off_host == nullptr)) return CHOL_ERR_ARG;
    if (batch == 0) return CHOL_OK;
    if (A_host == nullptr || X_host == nullptr || A_host == X_host) return CHOL_ERR_ARG;
    const bool sized = n_host != nullptr;
    const HostSlotLayout L = host_slot_layout(dt, batch, max_n, o.layout, sized);
    if (ws == nullptr || ws_bytes < L.bytes || reinterpret_cast<uintptr_t>(ws) % 256 != 0)
        return CHOL_ERR_WORKSPACE;
    if (o.layout == 0) o.fill_lower = 1;  // every element of a dense matrix goes back to the host
    const size_t es = elem_size(dt);
    const int64_t mc = host_chunk_matrices(batch);
    const int64_t nchunks = (batch + mc - 1) / mc;
    const int64_t cap = mc * matrix_elems(o.layout, max_n);
    // element span [e0, e1) of chunk k (matrices stored back to back in index order)
    auto span = [&](int64_t k, int64_t* e0, int64_t* e1) {
        const int64_t b0 = k * mc, b1 = std::min<int64_t>(b0 + mc, batch);
        if (!sized) {
            *e0 = b0 * matrix_elems(o.layout, max_n);
            *e1 = b1 * matrix_elems(o.layout, max_n);
        } else {
            const int32_t nl = std::min(std::max(n_host[b1 - 1], 0), max_n);
            *e0 = off_host[b0];
            *e1 = off_host[b1 - 1] + matrix_elems(o.layout, nl);
        }
    };
    for (int64_t k = 0; k < nchunks; ++k) {
        int64_t e0, e1;
        span(k, &e0, &e1);
        if (e0 < 0 || e1 < e0 || e1 - e0 > cap) return CHOL_ERR_ARG;  // not stored back to back
    }
    HostStreams* hs = host_streams();
    if (hs == nullptr) return CHOL_ERR_CUDA;
    std::lock_guard<std::mutex> lk(hs->mu);
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    cudaStream_t stage[4] = {hs->in, hs->run[0], hs->run[1], hs->out};
    if (cudaEventRecord(hs->fork, cs) != cudaSuccess) return CHOL_ERR_CUDA;
    for (cudaStream_t st2 : stage)
        if (cudaStreamWaitEvent(st2, hs->fork, 0) != cudaSuccess) return CHOL_ERR_CUDA;
    const char* Ah = static_cast<const char*>(A_host);
    char* Xh = static_cast<char*>(X_host);
    char* wsb = static_cast<char*>(ws);
    int32_t* n_dev = reinterpret_cast<int32_t*>(wsb + L.n);
    int64_t* off_dev = reinterpret_cast<int64_t*>(wsb + L.off);
    int32_t* info_dev = reinterpret_cast<int32_t*>(wsb + L.info);
    // the orders and offsets of the whole batch, ahead of the first chunk
    if (sized && (cudaMemcpyAsync(n_dev, n_host, (size_t)batch * sizeof(int32_t), cudaMemcpyHostToDevice, hs->in) !=
                      cudaSuccess ||
                  cudaMemcpyAsync(off_dev, off_host, (size_t)batch * sizeof(int64_t), cudaMemcpyHostToDevice,
                                  hs->in) != cudaSuccess))
        return CHOL_ERR_CUDA;
    for (int64_t k = 0; k < nchunks; ++k) {
        const int slot = (int)(k % kHostSlots);
        char* base = wsb + L.slots + (size_t)slot * L.total;
        const int64_t b0 = k * mc;
        const int32_t cnt = (int32_t)(std::min<int64_t>(b0 + mc, batch) - b0);
        int64_t e0, e1;
        span(k, &e0, &e1);
        // The chunk's first element sits `lead` bytes into its slot, lead being
        // the host address's offset from a kHostAlign boundary, so that the
        // copies start on such a boundary on both sides.  The copy in starts
        // lead bytes early (elements of earlier matrices of the same array,
        // never before its start); the copy out splits off the head up to the
        // first boundary instead, as the bytes before the chunk belong to
        // another chunk's results.  Per-matrix offsets stay absolute: the
        // device base is shifted so that base + off[b] lands in the slot.
        const size_t cstart = (size_t)(e0 * (int64_t)es);
        const size_t bytes = (size_t)(e1 - e0) * es;
        const size_t lead_a = std::min<size_t>((reinterpret_cast<uintptr_t>(Ah) + cstart) % kHostAlign, cstart);
        const size_t lead_x = (reinterpret_cast<uintptr_t>(Xh) + cstart) % kHostAlign;
        // copy in, once the chunk that last used this slot has been copied out
        if (k >= kHostSlots && cudaStreamWaitEvent(hs->in, hs->freed[slot], 0) != cudaSuccess) return CHOL_ERR_CUDA;
        if (cudaMemcpyAsync(base + L.a, Ah + cstart - lead_a, bytes + lead_a, cudaMemcpyHostToDevice, hs->in) !=
            cudaSuccess)
            return CHOL_ERR_CUDA;
        if (cudaEventRecord(hs->loaded[k], hs->in) != cudaSuccess) return CHOL_ERR_CUDA;
        // kernels
        // a chunk's kernels fill only part of the GPU: consecutive chunks run side by side
        cudaStream_t run = hs->run[k % 2];
        if (cudaStreamWaitEvent(run, hs->loaded[k], 0) != cudaSuccess) return CHOL_ERR_CUDA;
        const intptr_t shift = sized ? (intptr_t)cstart : 0;
        const void* Ad = reinterpret_cast<const void*>(reinterpret_cast<intptr_t>(base + L.a + lead_a) - shift);
        void* Xd = reinterpret_cast<void*>(reinterpret_cast<intptr_t>(base + L.x + lead_x) - shift);
        BatchParams p = make_params(cnt, sized ? n_dev + b0 : nullptr, sized ? off_dev + b0 : nullptr, max_n, Ad,
                                    nullptr, Xd, info_dev + b0, o, 1);
        // the orders are in host memory here: launch only the classes that occur
        // (an order outside [0, max_n] is left to the device check, which flags it)
        uint8_t present[kClasses] = {};
        if (sized)
            for (int32_t b = 0; b < cnt; ++b) {
                const uint32_t nb = (uint32_t)n_host[b0 + b];
                if (nb < (uint32_t)kClasses) present[nb] = 1;
            }
        st = enqueue_inv(dt, p, base + L.ws, run, false, o, sized ? present : nullptr);
        if (st != CHOL_OK) return st;
        if (cudaEventRecord(hs->computed[k], run) != cudaSuccess) return CHOL_ERR_CUDA;
        // copy out, then free the slot
        if (cudaStreamWaitEvent(hs->out, hs->computed[k], 0) != cudaSuccess) return CHOL_ERR_CUDA;
        const size_t head = std::min(bytes, (kHostAlign - lead_x) % kHostAlign);
        if (head > 0 &&
            cudaMemcpyAsync(Xh + cstart, base + L.x + lead_x, head, cudaMemcpyDeviceToHost, hs->out) != cudaSuccess)
            return CHOL_ERR_CUDA;
        if (bytes > head && cudaMemcpyAsync(Xh + cstart + head, base + L.x + lead_x + head, bytes - head,
                                            cudaMemcpyDeviceToHost, hs->out) != cudaSuccess)
            return CHOL_ERR_CUDA;
        if (cudaEventRecord(hs->freed[slot], hs->out) != cudaSuccess) return CHOL_ERR_CUDA;
    }
    // info of the whole batch, after the last chunk's kernels (the copy-out
    // stream has waited for them)
    if (info_host && cudaMemcpyAsync(info_host, info_dev, (size_t)batch * sizeof(int32_t), cudaMemcpyDeviceToHost,
                                     hs->out) != cudaSuccess)
        return CHOL_ERR_CUDA;
    for (int k = 0; k < 4; ++k)
        if (cudaEventRecord(hs->join[k], stage[k]) != cudaSuccess || cudaStreamWaitEvent(cs, hs->join[k], 0) != cudaSuccess)
            return CHOL_ERR_CUDA;
    return CHOL_OK;
}

size_t chol_workspace_bytes(int32_t call, chol_dtype_t dt, int32_t batch, int32_t max_n, int32_t has_sizes,
                            const chol_opts_t* opts) {
    const chol_opts_t o = opts_or_default(opts);
    if (call == CHOL_CALL_MMSE) {
        if (batch <= 0 || max_n < 1 || max_n > kBatchedMaxN || dt < CHOL_F32 || dt > CHOL_C128) return 0;
        return 2 * mmse_ws_matrices(dt, batch, max_n) + ws_need_batched(batch, has_sizes);
    }
    if (max_n > kBatchedMaxN && (call == CHOL_CALL_FACTOR || call == CHOL_CALL_INV))
        return blocked_workspace_bytes(dt, max_n, call == CHOL_CALL_INV ? blocked_refine_steps(o) : 0);
    if (call == CHOL_CALL_FACTOR || call == CHOL_CALL_INV) return ws_need_batched(batch, has_sizes);
    if (call == CHOL_CALL_INV_HOST) {
        if (batch <= 0 || max_n < 1 || max_n > kBatchedMaxN || dt < CHOL_F32 || dt > CHOL_C128) return 0;
        return host_slot_layout(dt, batch, max_n, o.layout, has_sizes != 0).bytes;
    }
    return 0;
}

const char* chol_status_string(chol_status_t status) {
    switch (status) {
        case CHOL_OK: return "success";
        case CHOL_ERR_ARG: return "invalid argument";
        case CHOL_ERR_CUDA: return "a CUDA runtime call failed";
        case CHOL_ERR_UNSUPPORTED: return "dtype, precision or size not supported";
        case CHOL_ERR_TIMEOUT: return "a bounded device wait gave up";
        case CHOL_ERR_WORKSPACE: return "workspace missing, too small or not 256-byte aligned";
    }
    return "unknown status";
}

chol_status_t chol_last_device_error(void* stream) {
    DevState* ds = nullptr;
    if (dev_state(&ds) != cudaSuccess) return CHOL_ERR_CUDA;
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return CHOL_ERR_CUDA;
    int v = 0;
    if (cudaMemcpy(&v, ds->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return CHOL_ERR_CUDA;
    if (v != 0) {
        const int z = 0;
        if (cudaMemcpy(ds->err, &z, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) return CHOL_ERR_CUDA;
    }
    return static_cast<chol_status_t>(v);
}

chol_status_t chol_mmse_batched(chol_dtype_t dt, int32_t batch, const int32_t* n, const int32_t* m,
                                const int64_t* hoff, const int64_t* woff, int32_t max_n, int32_t max_m, const void* H,
                                double sigma2, void* W, int32_t* info, const chol_opts_t* opts, void* ws,
                                size_t ws_bytes, void* stream) {
    chol_opts_t o = opts_or_default(opts);
    o.layout = 1;  // A and X live packed in the workspace
    o.fill_lower = 0;
    chol_status_t st = check_common(dt, batch, max_n, o);
    if (st != CHOL_OK || batch == 0) return st;
    if (max_m < 1 || !(sigma2 >= 0.0) || !std::isfinite(sigma2)) return CHOL_ERR_ARG;
    if (H == nullptr || W == nullptr) return CHOL_ERR_ARG;
    if ((o.flags & CHOL_FLAG_PIVOT64_AUTO) && info == nullptr) return CHOL_ERR_ARG;
    const size_t es = dt == CHOL_F32 ? 4 : dt == CHOL_C128 ? 16 : 8;
    if (((size_t)(max_m + 1) * max_n + (size_t)max_n * (max_n + 1)) * es > 98304) return CHOL_ERR_UNSUPPORTED;
    const size_t mats = mmse_ws_matrices(dt, batch, max_n);
    const size_t need = 2 * mats + ws_need_batched(batch, n != nullptr);
    if (ws == nullptr || ws_bytes < need || reinterpret_cast<uintptr_t>(ws) % 256 != 0) return CHOL_ERR_WORKSPACE;
    char* w = static_cast<char*>(ws);
    MmseParams mp;
    std::memset(&mp, 0, sizeof(mp));
    mp.batch = batch;
    mp.n = n;
    mp.m = m;
    mp.hoff = hoff;
    mp.woff = woff;
    mp.max_n = max_n;
    mp.max_m = max_m;
    mp.H = H;
    mp.A = w;
    mp.X = w + mats;
    mp.W = W;
    mp.info = info;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (launch_mmse(dt, 0, mp, sigma2, s, false) != cudaSuccess) return CHOL_ERR_CUDA;
    BatchParams p = make_params(batch, n, nullptr, max_n, mp.A, nullptr, mp.X, info, o, 1);
    st = enqueue_inv(dt, p, w + 2 * mats, s, false, o);
    if (st != CHOL_OK) return st;
    if (launch_mmse(dt, 1, mp, sigma2, s, false) != cudaSuccess) return CHOL_ERR_CUDA;
    return CHOL_OK;
}

chol_status_t chol_blocked_timing(int32_t enable) {
    if (enable != 0 && enable != 1) return CHOL_ERR_ARG;
    blocked_timing_enable(enable);
    return CHOL_OK;
}

chol_status_t chol_blocked_timing_read(int32_t kind, float* ms, double* flops, int32_t* launches) {
    if (ms == nullptr || flops == nullptr || launches == nullptr) return CHOL_ERR_ARG;
    int l = 0;
    const cudaError_t e = blocked_timing_read(kind, ms, flops, &l);
    *launches = l;
    if (e == cudaErrorInvalidValue) return CHOL_ERR_ARG;
    return e == cudaSuccess ? CHOL_OK : CHOL_ERR_CUDA;
}

chol_status_t chol_pivot64_redo_count(void* stream, int64_t* count) {
    if (count == nullptr) return CHOL_ERR_ARG;
    DevState* ds = nullptr;
    if (dev_state(&ds) != cudaSuccess) return CHOL_ERR_CUDA;
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return CHOL_ERR_CUDA;
    unsigned long long v = 0;
    if (cudaMemcpy(&v, ds->redo, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) return CHOL_ERR_CUDA;
    if (v != 0) {
        const unsigned long long z = 0;
        if (cudaMemcpy(ds->redo, &z, sizeof(z), cudaMemcpyHostToDevice) != cudaSuccess) return CHOL_ERR_CUDA;
    }
    *count = (int64_t)v;
    return CHOL_OK;
}

// ---------------------------------------------------------------------------
// chol_inv_batched_noalloc: the bucketing scratch of a batch with per-matrix
// sizes lives in this fixed device array instead of a caller workspace.
// ---------------------------------------------------------------------------
}  // extern "C"

namespace {
constexpr size_t kNoallocScratchBytes = kWsHeader + 4 * (size_t)CHOL_NOALLOC_MAX_BATCH;
}
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

namespace {
void* g_noalloc_ptr[kMaxDevices];
std::mutex g_noalloc_mu;

// Device address of g_noalloc_scratch on the current device, looked up once
// per device (host code cannot use the symbol itself as a device pointer).
chol_status_t noalloc_scratch(void** out) {
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess) return CHOL_ERR_CUDA;
    if (d < 0 || d >= kMaxDevices) return CHOL_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (g_noalloc_ptr[d] == nullptr) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return CHOL_ERR_CUDA;
        g_noalloc_ptr[d] = p;
    }
    *out = g_noalloc_ptr[d];
    return CHOL_OK;
}
}  // namespace

extern "C" {

chol_status_t chol_inv_batched_noalloc(chol_dtype_t dt, int32_t batch, const int32_t* n, const int64_t* off,
                                       int32_t max_n, const void* A, void* R, void* X, int32_t* info,
                                       const chol_opts_t* opts, void* stream) {
    const chol_opts_t o = opts_or_default(opts);
    chol_status_t st = check_common(dt, batch, max_n, o);
    if (st != CHOL_OK || batch == 0) return st;
    if (A == nullptr || X == nullptr) return CHOL_ERR_ARG;
    if (o.prec == CHOL_PREC_FP32_REFINE && o.refine_steps != 0 && X == A) return CHOL_ERR_ARG;
    if ((o.flags & CHOL_FLAG_PIVOT64_AUTO) && info == nullptr) return CHOL_ERR_ARG;
    if (n != nullptr && batch > CHOL_NOALLOC_MAX_BATCH) return CHOL_ERR_WORKSPACE;
    void* scratch = nullptr;
    if (n != nullptr) {
        st = noalloc_scratch(&scratch);
        if (st != CHOL_OK) return st;
    }
    BatchParams p = make_params(batch, n, off, max_n, A, (R == X) ? nullptr : R, X, info, o, 1);
    return enqueue_inv(dt, p, scratch, static_cast<cudaStream_t>(stream), false, o);
}

int32_t chol_version(void) { return 100; }

chol_status_t chol_plan_inv_create(chol_plan_t** plan, chol_dtype_t dt, int32_t batch, const int32_t* n,
                                   const int64_t* off, int32_t max_n, const void* A, void* R, void* X,
                                   int32_t* info, const chol_opts_t* opts, void* ws, size_t ws_bytes) {
    if (plan == nullptr) return CHOL_ERR_ARG;
    *plan = nullptr;
    chol_opts_t o = opts_or_default(opts);
    const bool timed = (o.flags & CHOL_FLAG_PLAN_TIMING) != 0;
    const bool fixed_orders = (o.flags & CHOL_FLAG_PLAN_ORDERS) != 0;
    o.flags &= ~(CHOL_FLAG_PLAN_TIMING | CHOL_FLAG_PLAN_ORDERS);
    chol_status_t st = inv_validate(dt, batch, n, max_n, A, X, info, o, ws, ws_bytes);
    if (st != CHOL_OK) return st;
    BatchParams p = make_params(batch, n, off, max_n, A, (R == X) ? nullptr : R, X, info, o, 1);
    // CHOL_FLAG_PLAN_ORDERS: the orders present now (n read once, on the host)
    uint8_t present[kClasses] = {};
    const bool use_present = fixed_orders && n != nullptr && batch > 0 && max_n <= kBatchedMaxN;
    if (use_present) {
        std::vector<int32_t> nh((size_t)batch);
        if (cudaMemcpy(nh.data(), n, (size_t)batch * sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
            return CHOL_ERR_CUDA;
        const uint64_t stated[2] = {p.order_mask[0], p.order_mask[1]};
        p.order_mask[0] = p.order_mask[1] = 0;
        for (int32_t v : nh)
            if (v > 0 && v <= max_n && order_allowed(stated[0], stated[1], v)) {
                present[v] = 1;
                p.order_mask[v / 64] |= 1ull << (v % 64);
            }
    }
    // one-time kernel set-up outside the capture
    st = enqueue_inv(dt, p, ws, nullptr, true, o, use_present ? present : nullptr);
    if (st != CHOL_OK) return st;
    chol_plan* pl = new chol_plan();
    if (timed) {
        pl->timing = new ClassTiming();
        for (int c = 0; c < kClasses; ++c) {
            pl->timing->used[c] = false;
            if (cudaEventCreate(&pl->timing->start[c]) != cudaSuccess ||
                cudaEventCreate(&pl->timing->end[c]) != cudaSuccess) {
                delete pl->timing;
                delete pl;
                return CHOL_ERR_CUDA;
            }
        }
    }
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        chol_plan_destroy(pl);
        return CHOL_ERR_CUDA;
    }
    st = CHOL_OK;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) st = CHOL_ERR_CUDA;
    t_timing = pl->timing;
    if (st == CHOL_OK && batch > 0) st = enqueue_inv(dt, p, ws, cs, false, o, use_present ? present : nullptr);
    t_timing = nullptr;
    cudaGraph_t g = nullptr;
    if (cudaStreamEndCapture(cs, &g) != cudaSuccess && st == CHOL_OK) st = CHOL_ERR_CUDA;
    pl->graph = g;
    if (st == CHOL_OK && cudaGraphInstantiate(&pl->exec, g, 0) != cudaSuccess) st = CHOL_ERR_CUDA;
    cudaStreamDestroy(cs);
    if (st != CHOL_OK) {
        chol_plan_destroy(pl);
        return st;
    }
    *plan = pl;
    return CHOL_OK;
}

chol_status_t chol_plan_launch(chol_plan_t* plan, void* stream) {
    if (plan == nullptr || plan->exec == nullptr) return CHOL_ERR_ARG;
    if (cudaGraphLaunch(plan->exec, static_cast<cudaStream_t>(stream)) != cudaSuccess) return CHOL_ERR_CUDA;
    return CHOL_OK;
}

chol_status_t chol_plan_destroy(chol_plan_t* plan) {
    if (plan == nullptr) return CHOL_ERR_ARG;
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    if (plan->graph) cudaGraphDestroy(plan->graph);
    if (plan->timing) {
        for (int c = 0; c < kClasses; ++c) {
            cudaEventDestroy(plan->timing->start[c]);
            cudaEventDestroy(plan->timing->end[c]);
        }
        delete plan->timing;
    }
    delete plan;
    return CHOL_OK;
}

chol_status_t chol_plan_kernel_ms(chol_plan_t* plan, int32_t order, float* ms) {
    if (plan == nullptr || ms == nullptr || plan->timing == nullptr) return CHOL_ERR_ARG;
    if (order < 0 || order >= kClasses || !plan->timing->used[order]) return CHOL_ERR_ARG;
    if (cudaEventElapsedTime(ms, plan->timing->start[order], plan->timing->end[order]) != cudaSuccess)
        return CHOL_ERR_CUDA;
    return CHOL_OK;
}

}  // extern "C"
