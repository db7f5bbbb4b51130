// Register-tiled products of two square tiles in shared memory on one warp:
// each lane holds a block of the product and walks k over the squares' rows,
// so one shared load feeds several multiply-adds.  Used by the adjoint (order
// 32 squares) and the refinement (order 16 or 32) of orders up to 32, the
// matrices zero-padded to the square.
#pragma once

#include <type_traits>

#include "batched.cuh"

namespace cholinv {

constexpr int kTB = 32;          // padded order of the adjoint's squares
constexpr int kTLD = kTB + 4;    // row stride

// Squares of order TB (16 or 32) in shared memory with row stride TB + 4;
// lane l of a warp holds the TR x TC block at rows TR (l / 4).., columns
// TC (l % 4).. (eight row groups by four column groups).
template <int TB>
struct Tile {
    static_assert(TB == 16 || TB == 32, "square tiles of order 16 or 32");
    static constexpr int LD = TB + 4;
    static constexpr int TR = TB / 8;
    static constexpr int TC = TB / 4;
};

// acc[r][c] += sum_k op(Lt[k][r0 + r]) Rm[k][c0 + c], k = 0..TB-1; op is the
// conjugate when CONJ.  FP32 and complex64 run on paired FP32 instructions
// (two entries of a row, or the two parts of a complex entry, per
// instruction); FP64 types on plain fused multiply-adds.
template <typename V, bool CONJ, int TB = kTB>
CHOL_D void tile_product(const V* Lt, const V* Rm, int r0, int c0, V (&acc)[Tile<TB>::TR][Tile<TB>::TC]) {
    constexpr int LD = Tile<TB>::LD, TR = Tile<TB>::TR, TC = Tile<TB>::TC;
    if constexpr (std::is_same<V, float>::value) {
        float2 a2[TR][TC / 2];
#pragma unroll
        for (int r = 0; r < TR; ++r)
#pragma unroll
            for (int cp = 0; cp < TC / 2; ++cp) a2[r][cp] = make_float2(acc[r][2 * cp], acc[r][2 * cp + 1]);
#pragma unroll 4
        for (int k = 0; k < TB; ++k) {
            float2 b[TC / 2];
#pragma unroll
            for (int cp = 0; cp < TC / 2; ++cp) b[cp] = *reinterpret_cast<const float2*>(&Rm[k * LD + c0 + 2 * cp]);
#pragma unroll
            for (int r = 0; r < TR; ++r) {
                const float a = Lt[k * LD + r0 + r];
                const float2 aa = make_float2(a, a);
#pragma unroll
                for (int cp = 0; cp < TC / 2; ++cp) a2[r][cp] = __ffma2_rn(aa, b[cp], a2[r][cp]);
            }
        }
#pragma unroll
        for (int r = 0; r < TR; ++r)
#pragma unroll
            for (int cp = 0; cp < TC / 2; ++cp) {
                acc[r][2 * cp] = a2[r][cp].x;
                acc[r][2 * cp + 1] = a2[r][cp].y;
            }
        return;
    } else if constexpr (std::is_same<V, cpx<float>>::value) {
        // {re, im} += a.re {b.re, b.im} + a.im {-b.im, b.re}  (a conjugated when CONJ)
#pragma unroll 2
        for (int k = 0; k < TB; ++k) {
            float2 b[TC], bs[TC];
#pragma unroll
            for (int c = 0; c < TC; ++c) {
                const cpx<float> v = Rm[k * LD + c0 + c];
                b[c] = make_float2(v.re, v.im);
                bs[c] = make_float2(-v.im, v.re);
            }
#pragma unroll
            for (int r = 0; r < TR; ++r) {
                const cpx<float> a = Lt[k * LD + r0 + r];
                const float ai = CONJ ? -a.im : a.im;
                const float2 ar = make_float2(a.re, a.re), aim = make_float2(ai, ai);
#pragma unroll
                for (int c = 0; c < TC; ++c) {
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
    for (int k = 0; k < TB; ++k) {
        V a[TR], b[TC];
#pragma unroll
        for (int r = 0; r < TR; ++r) a[r] = CONJ ? conj_v(Lt[k * LD + r0 + r]) : Lt[k * LD + r0 + r];
#pragma unroll
        for (int c = 0; c < TC; ++c) b[c] = Rm[k * LD + c0 + c];
#pragma unroll
        for (int r = 0; r < TR; ++r)
#pragma unroll
            for (int c = 0; c < TC; ++c) acc[r][c] = fma_v(a[r], b[c], acc[r][c]);
    }
}

}  // namespace cholinv
