// Shared device-side types and helpers of the cholinv CUDA library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cholinv.h"

#define CHOL_HD __host__ __device__ __forceinline__
#define CHOL_CX __host__ __device__ __forceinline__ constexpr
#define CHOL_D __device__ __forceinline__

namespace cholinv {

// ---------------------------------------------------------------------------
// Value types: real float/double and an interleaved complex pair.
// ---------------------------------------------------------------------------
template <typename T>
struct __align__(2 * sizeof(T)) cpx {
    T re, im;
};

template <typename V> struct traits;
template <> struct traits<float>        { using real = float;  static constexpr bool cplx = false; static constexpr int words = 1; };
template <> struct traits<double>       { using real = double; static constexpr bool cplx = false; static constexpr int words = 2; };
template <> struct traits<cpx<float>>   { using real = float;  static constexpr bool cplx = true;  static constexpr int words = 2; };
template <> struct traits<cpx<double>>  { using real = double; static constexpr bool cplx = true;  static constexpr int words = 4; };

template <typename T> CHOL_HD T zero_v() { return T(0); }
template <> CHOL_HD cpx<float> zero_v<cpx<float>>() { return {0.f, 0.f}; }
template <> CHOL_HD cpx<double> zero_v<cpx<double>>() { return {0.0, 0.0}; }

// real part, conjugate, |v|^2
CHOL_HD float re_of(float v) { return v; }
CHOL_HD double re_of(double v) { return v; }
template <typename T> CHOL_HD T re_of(cpx<T> v) { return v.re; }

CHOL_HD float conj_v(float v) { return v; }
CHOL_HD double conj_v(double v) { return v; }
template <typename T> CHOL_HD cpx<T> conj_v(cpx<T> v) { return {v.re, -v.im}; }

template <typename T> CHOL_HD cpx<T> operator+(cpx<T> a, cpx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T> CHOL_HD cpx<T> operator-(cpx<T> a, cpx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T> CHOL_HD cpx<T> operator*(cpx<T> a, T s) { return {a.re * s, a.im * s}; }
template <typename T> CHOL_HD cpx<T> operator-(cpx<T> a) { return {-a.re, -a.im}; }

// acc + a*b with fused multiply-adds (real: 1 FMA; complex: 4 FMAs)
CHOL_D float fma_v(float a, float b, float acc) { return fmaf(a, b, acc); }
CHOL_D double fma_v(double a, double b, double acc) { return fma(a, b, acc); }
template <typename T> CHOL_D cpx<T> fma_v(cpx<T> a, cpx<T> b, cpx<T> acc) {
    cpx<T> r;
    r.re = fma(a.re, b.re, acc.re);
    r.re = fma(-a.im, b.im, r.re);
    r.im = fma(a.re, b.im, acc.im);
    r.im = fma(a.im, b.re, r.im);
    return r;
}
// acc - conj(a)*b
CHOL_D float fnma_conj(float a, float b, float acc) { return fmaf(-a, b, acc); }
CHOL_D double fnma_conj(double a, double b, double acc) { return fma(-a, b, acc); }
template <typename T> CHOL_D cpx<T> fnma_conj(cpx<T> a, cpx<T> b, cpx<T> acc) {
    // conj(a)*b = (ar*br + ai*bi) + i(ar*bi - ai*br)
    cpx<T> r;
    r.re = fma(-a.re, b.re, acc.re);
    r.re = fma(-a.im, b.im, r.re);
    r.im = fma(-a.re, b.im, acc.im);
    r.im = fma(a.im, b.re, r.im);
    return r;
}
// acc + a*conj(b)
CHOL_D float fma_conjb(float a, float b, float acc) { return fmaf(a, b, acc); }
CHOL_D double fma_conjb(double a, double b, double acc) { return fma(a, b, acc); }
template <typename T> CHOL_D cpx<T> fma_conjb(cpx<T> a, cpx<T> b, cpx<T> acc) {
    // a*conj(b) = (ar*br + ai*bi) + i(ai*br - ar*bi)
    cpx<T> r;
    r.re = fma(a.re, b.re, acc.re);
    r.re = fma(a.im, b.im, r.re);
    r.im = fma(a.im, b.re, acc.im);
    r.im = fma(-a.re, b.im, r.im);
    return r;
}
// Re(a * conj(b)) accumulated into a real accumulator
CHOL_D float fma_re_conjb(float a, float b, float acc) { return fmaf(a, b, acc); }
CHOL_D double fma_re_conjb(double a, double b, double acc) { return fma(a, b, acc); }
template <typename T> CHOL_D T fma_re_conjb(cpx<T> a, cpx<T> b, T acc) {
    return fma(a.im, b.im, fma(a.re, b.re, acc));
}
// acc - |a|^2 (real accumulator)
CHOL_D float fnma_abs2(float a, float acc) { return fmaf(-a, a, acc); }
CHOL_D double fnma_abs2(double a, double acc) { return fma(-a, a, acc); }
template <typename T> CHOL_D T fnma_abs2(cpx<T> a, T acc) { return fma(-a.im, a.im, fma(-a.re, a.re, acc)); }

CHOL_D float scale_v(float v, float s) { return v * s; }
CHOL_D double scale_v(double v, double s) { return v * s; }
template <typename T> CHOL_D cpx<T> scale_v(cpx<T> v, T s) { return {v.re * s, v.im * s}; }

template <typename V> CHOL_D V from_real(typename traits<V>::real r);
template <> CHOL_D float from_real<float>(float r) { return r; }
template <> CHOL_D double from_real<double>(double r) { return r; }
template <> CHOL_D cpx<float> from_real<cpx<float>>(float r) { return {r, 0.f}; }
template <> CHOL_D cpx<double> from_real<cpx<double>>(double r) { return {r, 0.0}; }

template <typename V> CHOL_D V nan_v() {
    using R = typename traits<V>::real;
    R q = R(__int_as_float(0x7fffffff));
    if constexpr (traits<V>::cplx) return V{q, q}; else return V(q);
}

template <typename R> CHOL_D bool pivot_ok(R t) { return (t > R(0)) && isfinite(t); }

// r_ii = sqrt(t) and 1/r_ii from Eq. 3's argument t.  FP32: the hardware
// reciprocal square root y refined by one Newton step written around its
// residual, e = 1 - (t y) y (one fused multiply-add), y <- y + (y/2) e, which
// keeps 1/r_ii within an ulp (a correctly rounded sqrt followed by a
// correctly rounded divide can be 1.5 ulp off) at a fraction of their
// instructions; then r_ii = t y.  FP64: sqrt and divide.
CHOL_D void pivot_root(float t, float& rii, float& inv) {
    const float y = rsqrtf(t);
    const float e = fmaf(-(t * y), y, 1.0f);
    inv = fmaf(0.5f * y, e, y);
    rii = t * inv;
}
CHOL_D void pivot_root(double t, double& rii, double& inv) {
    rii = sqrt(t);
    inv = 1.0 / rii;
}

// Eq. 3's root from an argument t accumulated in FP64 (FP64 pivots), for a
// factor held in R: r_ii = sqrt(t) and 1/r_ii.  For FP32 factors the
// hardware FP32 reciprocal square root of t is refined by one
// Newton-Raphson step taken in FP64 arithmetic, y <- y + (y/2)(1 - t y^2),
// good to about 44 bits before the rounding to FP32 (the FP64 square root
// and division are long instruction sequences on the FP64 pipe); outside the
// normal FP32 range of t, and for FP64 factors, the FP64 square root and
// division.
template <typename R>
CHOL_D void pivot_root64(double t, R& rii, R& inv) {
    if constexpr (sizeof(R) == 4) {
        if (t >= 1.2e-38 && t <= 3.0e38) {
            const double y = (double)rsqrtf((float)t);
            const double e = fma(-(t * y), y, 1.0);
            const double yi = fma(0.5 * y, e, y);
            inv = (R)yi;
            rii = (R)(t * yi);
            return;
        }
    }
    const double r = sqrt(t);
    rii = (R)r;
    inv = (R)(1.0 / r);
}

// ---------------------------------------------------------------------------
// Compensated FP32 accumulation (Ogita, Rump & Oishi, "Accurate sum and dot
// product", 2005, Algorithm Dot2): a dot product carried as an unevaluated
// pair s + c.  Each product a b is split exactly into p = fl(a b) and its
// rounding error fma(a, b, -p); each sum s + p into fl(s + p) and its
// rounding error (Knuth's TwoSum); the errors accumulate in c.  The result
// is as accurate as a dot product in twice FP32's precision (about 48
// bits).  The _rn intrinsics keep the compiler from contracting or
// reassociating any of the steps.
// ---------------------------------------------------------------------------
struct f2acc {
    float s, c;
};
CHOL_D f2acc f2_init(float v) { return {v, 0.f}; }
// r += a b
CHOL_D void f2_fma(f2acc& r, float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    const float t = __fadd_rn(r.s, p);
    const float z = __fsub_rn(t, r.s);
    const float err = __fadd_rn(__fsub_rn(r.s, __fsub_rn(t, z)), __fsub_rn(p, z));
    r.s = t;
    r.c = __fadd_rn(r.c, __fadd_rn(err, e));
}
CHOL_D float f2_value(const f2acc& r) { return __fadd_rn(r.s, r.c); }

// The same on two independent dot products at once (paired FP32
// instructions, sm_100 and later): lanes x and y of every float2.
struct f2acc2 {
    float2 s, c;
};
CHOL_D float2 neg2(float2 v) { return make_float2(-v.x, -v.y); }
// r += a b, lane by lane
CHOL_D void f2_fma2(f2acc2& r, float2 a, float2 b) {
    const float2 p = __fmul2_rn(a, b);
    const float2 e = __ffma2_rn(a, b, neg2(p));
    const float2 t = __fadd2_rn(r.s, p);
    const float2 z = __fadd2_rn(t, neg2(r.s));
    const float2 err = __fadd2_rn(__fadd2_rn(r.s, neg2(__fadd2_rn(t, neg2(z)))), __fadd2_rn(p, neg2(z)));
    r.s = t;
    r.c = __fadd2_rn(r.c, __fadd2_rn(err, e));
}

// ---------------------------------------------------------------------------
// Index helpers.  Packed upper, row by row: row i holds columns i..n-1.
// ---------------------------------------------------------------------------
CHOL_CX int pidx(int n, int i, int j) { return i * n - (i * (i - 1)) / 2 + (j - i); }

// Row and column (i <= j) of element e of an order-n packed upper triangle:
// i from the closed form of pidx's inverse, corrected by one step either way
// against rounding.
CHOL_D void tri_rc(int n, int e, int& i, int& j) {
    const float b = 2.0f * n + 1.0f;
    int r = (int)((b - sqrtf(b * b - 8.0f * (float)e)) * 0.5f);
    r = max(0, min(r, n - 1));
    if (pidx(n, r, r) > e) --r;
    else if (r + 1 < n && pidx(n, r + 1, r + 1) <= e) ++r;
    i = r;
    j = e - pidx(n, r, r) + r;
}
CHOL_CX int tri(int n) { return n * (n + 1) / 2; }
CHOL_CX int64_t tri64(int64_t n) { return n * (n + 1) / 2; }

// element offset of (i,j), i <= j, within one matrix of order n
CHOL_HD int64_t elem_off(int layout, int n, int i, int j) {
    return layout ? (int64_t)pidx(n, i, j) : (int64_t)i * n + j;
}

// Kernels that detect an invalid input record the first error code in a
// per-device error word whose address they receive as an argument.
CHOL_D void report_error(int* err, int code) {
    if (err) atomicCAS(err, 0, code);
}

}  // namespace cholinv
