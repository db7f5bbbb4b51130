// Host-side launchers of the batched kernels for one value type.  Each
// dtype's translation unit includes this file and instantiates
// launch_batched<V> (four TUs compile in parallel).
#pragma once

#include <algorithm>
#include <mutex>
#include <type_traits>

#include "batched.cuh"
#include "dispatch.h"
#include "group.cuh"

namespace cholinv {

// Kernel family per order N:
//   lane  (one matrix per thread) while the packed triangle fits registers,
//   group (G threads per matrix) up to order 32 when a G <= 32 fits,
//   warp  (one matrix per warp, matrix in shared memory) otherwise.
constexpr int kGroupMaxN = 32;
template <typename V, int N>
constexpr int kernel_kind() {  // 0 lane, 1 group, 2 warp
    return LaneCfg<V, N>::REGS ? 0 : (N <= kGroupMaxN && group_size<V, N>() > 0) ? 1 : 2;
}

// CHOL_FLAG_PIVOT64_AUTO's FP32 pass: the kernels compiled with the
// cancellation test (GATE = true; FP32 value types), default variants only.
template <typename V>
CHOL_HD bool gate_on(const BatchParams& p) {
    return sizeof(typename traits<V>::real) == 4 && (p.flags & CHOL_FLAG_PIVOT64_AUTO) &&
           !(p.flags & CHOL_FLAG_PIVOT64);
}
template <typename V>
constexpr bool gate_built() { return sizeof(typename traits<V>::real) == 4; }

template <typename V, int N, bool GATE, bool LDL = false, bool P64 = false>
static cudaError_t launch_lane_t(const BatchParams& p, int upper_count, cudaStream_t s, bool dry) {
    constexpr int THREADS = LaneCfg<V, N>::THREADS;
    constexpr size_t SMEM = LaneCfg<V, N>::SMEM;
    auto kern = k_lane<V, N, GATE, LDL, P64>;
    static std::once_flag once;
    static int per_sm = 1;
    static cudaError_t setup_err = cudaSuccess;
    std::call_once(once, [&] {
        setup_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
        if (setup_err == cudaSuccess)
            setup_err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, SMEM);
        if (per_sm < 1) per_sm = 1;
    });
    if (setup_err != cudaSuccess || dry) return setup_err;
    const int chunks = (upper_count + THREADS - 1) / THREADS;
    if (chunks <= 0) return cudaSuccess;
    const int grid = std::min(chunks, device_info().sms * per_sm);
    kern<<<grid, THREADS, SMEM, s>>>(p);
    return cudaGetLastError();
}

template <typename V, int N>
static cudaError_t launch_lane(const BatchParams& p, int upper_count, cudaStream_t s, bool dry) {
    if constexpr (gate_built<V>())
        if (gate_on<V>(p)) return launch_lane_t<V, N, true>(p, upper_count, s, dry);
    return launch_lane_t<V, N, false>(p, upper_count, s, dry);
}

template <typename V>
static cudaError_t launch_warp(const BatchParams& p, int N, int upper_count, cudaStream_t s, bool dry) {
    const size_t per_warp = warp_elems(p, N) * sizeof(V);
    int warps = (int)std::max<size_t>(1, std::min<size_t>(4, 98304 / per_warp));
    const size_t smem = per_warp * warps;
    static std::once_flag once;
    static cudaError_t setup_err = cudaSuccess;
    std::call_once(once, [&] {
        setup_err = cudaFuncSetAttribute(k_warp<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    });
    if (setup_err != cudaSuccess || dry) return setup_err;
    int per_sm = 1;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_warp<V>, 32 * warps, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const int ctas = (upper_count + warps - 1) / warps;
    if (ctas <= 0) return cudaSuccess;
    const int grid = std::min(ctas, device_info().sms * per_sm);
    k_warp<V><<<grid, 32 * warps, smem, s>>>(p, N, warps);
    return cudaGetLastError();
}

// W warps per CTA; MINB resident CTAs per SM requested from the register
// allocator (MINB = 2 with W = 8 caps a thread at 128 registers).
template <typename V, int N, int G, int ALG, int W = 4, int MINB = 1, bool GATE = false, bool LDL = false,
          bool P64 = false>
static cudaError_t launch_group(const BatchParams& p, int upper_count, cudaStream_t s, bool dry) {
    using C = GroupCfg<V, N, G, W>;
    auto kern = k_group<V, N, G, ALG, W, MINB, GATE, LDL, P64>;
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

// Kernel variants of one order, chosen at run time by the autotuner
// (tune.cu) through variant_of(); variant 0 is the compiled-in default.
//   lane orders  : 0 lane; 1 group G=2 (orders >= 8 only)
//   group orders : 0 group G0; 1 group 2*G0 (when 2*G0 <= 32) in 256-thread
//                  CTAs capped at 128 registers per thread (two CTAs per SM)
//   warp orders  : 0 warp
template <typename V, int N>
constexpr int num_variants() {
    constexpr int kind = kernel_kind<V, N>();
    if constexpr (kind == 0) return (N >= 8 && N <= kGroupMaxN && group_size<V, N>() == 2) ? 2 : 1;
    else if constexpr (kind == 1) return group_size<V, N>() * 2 <= 32 ? 2 : 1;
    else return 1;
}

template <typename V, int N>
static cudaError_t launch_fixed(const BatchParams& p, int variant, int upper_count, cudaStream_t s, bool dry) {
    constexpr int kind = kernel_kind<V, N>();
    // the LDL form (CHOL_FLAG_LDL), FP64 pivots (CHOL_FLAG_PIVOT64) and the
    // cancellation test (CHOL_FLAG_PIVOT64_AUTO) run the default variant,
    // built for each
    if (p.flags & CHOL_FLAG_LDL) {
        if constexpr (kind == 0) return launch_lane_t<V, N, false, true>(p, upper_count, s, dry);
        else if constexpr (kind == 1)
            return launch_group<V, N, group_size<V, N>(), 1, 4, 1, false, true>(p, upper_count, s, dry);
        else return launch_warp<V>(p, N, upper_count, s, dry);
    }
    if constexpr (gate_built<V>()) {
        if (p.flags & CHOL_FLAG_PIVOT64) {
            if constexpr (kind == 0) return launch_lane_t<V, N, false, false, true>(p, upper_count, s, dry);
            else if constexpr (kind == 1)
                return launch_group<V, N, group_size<V, N>(), 1, 4, 1, false, false, true>(p, upper_count, s, dry);
            else return launch_warp<V>(p, N, upper_count, s, dry);
        }
    }
    if constexpr (kind == 0) {
        if constexpr (num_variants<V, N>() > 1)
            if (variant == 1 && !gate_on<V>(p)) return launch_group<V, N, 2, 1>(p, upper_count, s, dry);
        return launch_lane<V, N>(p, upper_count, s, dry);
    } else if constexpr (kind == 1) {
        constexpr int G0 = group_size<V, N>();
        if constexpr (gate_built<V>())
            if (gate_on<V>(p)) return launch_group<V, N, G0, 1, 4, 1, true>(p, upper_count, s, dry);
        if constexpr (num_variants<V, N>() > 1)
            if (variant == 1) return launch_group<V, N, (G0 * 2 <= 32 ? G0 * 2 : G0), 1, 8, 2>(p, upper_count, s, dry);
        return launch_group<V, N, G0, 1>(p, upper_count, s, dry);
    } else {
        return launch_warp<V>(p, N, upper_count, s, dry);
    }
}

// Launch class `cls` if it lies in [LO, N] (compile-time recursion).
template <typename V, int LO, int N>
static cudaError_t launch_fixed_range(const BatchParams& p, int cls, int variant, int upper_count, cudaStream_t s,
                                      bool dry) {
    if constexpr (N < LO) {
        return cudaErrorInvalidValue;
    } else {
        if (cls == N) return launch_fixed<V, N>(p, variant, upper_count, s, dry);
        return launch_fixed_range<V, LO, N - 1>(p, cls, variant, upper_count, s, dry);
    }
}

template <typename V, int LO, int N>
static int variants_range(int cls) {
    if constexpr (N < LO) {
        return 1;
    } else {
        if (cls == N) return num_variants<V, N>();
        return variants_range<V, LO, N - 1>(cls);
    }
}

template <typename V> constexpr int dtype_code();
template <> constexpr int dtype_code<float>() { return CHOL_F32; }
template <> constexpr int dtype_code<double>() { return CHOL_F64; }
template <> constexpr int dtype_code<cpx<float>>() { return CHOL_C64; }
template <> constexpr int dtype_code<cpx<double>>() { return CHOL_C128; }

// The orders of each element type are split over translation units that
// compile in parallel: [1, 14], [15, 20], [21, 25], [26, 29] and [30, 32]
// (kClassRanges; the last also takes the orders above 32).
// FP32 orders 33..64 (kWideLo..kWideHi in wide.cuh): variant 0 is the
// register-resident one-warp-per-matrix kernel (k_wide, in its own
// translation units), variant 1 the shared-memory warp kernel.  FP64 pivots
// on request (CHOL_FLAG_PIVOT64) run on the warp kernel.
constexpr int kWideMinN = 33;

// Launch the kernel of one size class (cls, in [LO, HI], or above
// kGroupMaxN when HI == kGroupMaxN) whose member count is at most
// upper_count, in the variant the tuning table holds for it.
template <typename V, int LO, int HI>
cudaError_t launch_class_range(const BatchParams& p, int cls, int upper_count, cudaStream_t s, bool dry) {
    // the comparison methods, and the LDL form above order 32, run on the warp kernel
    if ((p.flags & (CHOL_FLAG_METHOD_ES | CHOL_FLAG_METHOD_TMO)) || ((p.flags & CHOL_FLAG_LDL) && cls > kGroupMaxN))
        return launch_warp<V>(p, cls, upper_count, s, dry);
    const int v = variant_of(dtype_code<V>(), cls);
    if constexpr (HI == kGroupMaxN) {
        if (cls > kGroupMaxN) {
            if constexpr (std::is_same<V, float>::value)
                if (cls >= kWideMinN && (v == 0 || gate_on<V>(p)) && !(p.flags & CHOL_FLAG_PIVOT64))
                    return launch_wide_f32(p, cls, upper_count, s, dry);
            return launch_warp<V>(p, cls, upper_count, s, dry);
        }
    }
    return launch_fixed_range<V, LO, HI>(p, cls, v, upper_count, s, dry);
}

template <typename V, int LO, int HI>
int class_variants_range(int cls) {
    if (cls > kGroupMaxN) return (std::is_same<V, float>::value && cls >= kWideMinN) ? 2 : 1;
    return variants_range<V, LO, HI>(cls);
}

}  // namespace cholinv
