// Register-tiled products of two 32 x 32 squares in shared memory (row
// stride kTLD = 36) on one warp: lane l holds the 4 x 8 block at rows
// 4 (l / 4).., columns 8 (l % 4).., and walks k over the squares' rows, so
// one shared load feeds several multiply-adds.  Used by the adjoint and the
// refinement of orders up to 32 (zero-padded to 32).
#pragma once

#include <type_traits>

#include "batched.cuh"

namespace cholinv {

constexpr int kTB = 32;          // padded order
constexpr int kTLD = kTB + 4;    // row stride

// acc[r][c] += sum_k op(Lt[k][r0 + r]) Rm[k][c0 + c], k = 0..31; op is the
// conjugate when CONJ.  FP32 and complex64 run on paired FP32 instructions
// (two entries of a row, or the two parts of a complex entry, per
// instruction); FP64 types on plain fused multiply-adds.
template <typename V, bool CONJ>
CHOL_D void tile_product(const V* Lt, const V* Rm, int r0, int c0, V (&acc)[4][8]) {
    if constexpr (std::is_same<V, float>::value) {
        float2 a2[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int cp = 0; cp < 4; ++cp) a2[r][cp] = make_float2(acc[r][2 * cp], acc[r][2 * cp + 1]);
#pragma unroll 4
        for (int k = 0; k < kTB; ++k) {
            float2 b[4];
#pragma unroll
            for (int cp = 0; cp < 4; ++cp) b[cp] = *reinterpret_cast<const float2*>(&Rm[k * kTLD + c0 + 2 * cp]);
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const float a = Lt[k * kTLD + r0 + r];
                const float2 aa = make_float2(a, a);
#pragma unroll
                for (int cp = 0; cp < 4; ++cp) a2[r][cp] = __ffma2_rn(aa, b[cp], a2[r][cp]);
            }
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int cp = 0; cp < 4; ++cp) {
                acc[r][2 * cp] = a2[r][cp].x;
                acc[r][2 * cp + 1] = a2[r][cp].y;
            }
        return;
    } else if constexpr (std::is_same<V, cpx<float>>::value) {
        // {re, im} += a.re {b.re, b.im} + a.im {-b.im, b.re}  (a conjugated when CONJ)
#pragma unroll 2
        for (int k = 0; k < kTB; ++k) {
            float2 b[8], bs[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const cpx<float> v = Rm[k * kTLD + c0 + c];
                b[c] = make_float2(v.re, v.im);
                bs[c] = make_float2(-v.im, v.re);
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const cpx<float> a = Lt[k * kTLD + r0 + r];
                const float ai = CONJ ? -a.im : a.im;
                const float2 ar = make_float2(a.re, a.re), aim = make_float2(ai, ai);
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    float2 q = make_float2(acc[r][c].re, acc[r][c].im);
                    q = __ffma2_rn(ar, b[c], q);
                    q = __ffma2_rn(aim, bs[c], q);
                    acc[r][c] = {q.x, q.y};
                }
            }
        }
        return;
    }
#pragma unroll 4
    for (int k = 0; k < kTB; ++k) {
        V a[4], b[8];
#pragma unroll
        for (int r = 0; r < 4; ++r) a[r] = CONJ ? conj_v(Lt[k * kTLD + r0 + r]) : Lt[k * kTLD + r0 + r];
#pragma unroll
        for (int c = 0; c < 8; ++c) b[c] = Rm[k * kTLD + c0 + c];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[r][c] = fma_v(a[r], b[c], acc[r][c]);
    }
}

}  // namespace cholinv
