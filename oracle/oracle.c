/*
 * CPU oracle for "Matrix Inversion Using Cholesky Decomposition"
 * (Krishnamoorthy & Menon, arXiv 1111.4144).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * reference that the GPU library is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark load it.  It
 * shares no code, header, table or helper with the CUDA library, and the CUDA
 * library never calls it.
 *
 * Arithmetic: IEEE binary64 (complex: a pair of binary64), round to nearest,
 * correctly rounded sqrt and division, no fused multiply-add (the build passes
 * -ffp-contract=off).  Every sum runs with its index ascending.  Matrices are
 * dense, row-major, N x N.  Complex numbers are stored interleaved (re, im).
 * Only the upper triangle (i <= j) of an input Hermitian matrix is read; the
 * diagonal's imaginary part is ignored (a Hermitian diagonal is real).
 *
 * Functions and the passages they follow:
 *   orc_chol_{d,z}      Cholesky A = R^* R, row by row        Sec. II, Eqs. 2-4
 *   orc_inv_rows_{d,z}  proposed inverse R X = S, rows N..1   Sec. IV.A, Eqs. 20-24
 *   orc_inv_cols_{d,z}  same solve taken column by column     Sec. IV.A ("R x_i = s_i")
 *   orc_es_{d,z}        existing method "Equation Solving"    Sec. III.A, Eq. 15
 *   orc_tmo_{d,z}       existing "Triangular Matrix Ops"      Sec. III.B, Eqs. 16-19
 *   orc_ldl_{d,z}       LDL decomposition A = R^* D R         Sec. II.A, Eqs. 9-11
 *   orc_ldl_inv_{d,z}   proposed inverse via LDL              Sec. IV.B, Eqs. 25-29
 *   orc_gj_{ld,lz}      Gauss-Jordan in long double (an independent method, not in the paper)
 *   orc_grad_{d,z}      dA = -X sym(G) X (adjoint of the inverse; not in the paper)
 *   orc_inv_batch       batched driver over per-matrix sizes/offsets (threads over matrices)
 *   orc_chol_mt_d       orc_chol_d for one large matrix, the entries of each row split over threads
 *   orc_inv_rows_mt_d   orc_inv_rows_d for one large matrix, the same way
 *   orc_solve_cols_d    chosen columns of A^{-1} by the two triangular solves of Eq. 15
 *                       (R^* y = e_j, then R x = y), every row of each column, threads over columns
 *
 * Multiply counting (Table 1): every function that takes a `long long* mults`
 * adds one for each multiply inside an inner sum (a complex multiply counts as
 * one).  Square roots, reciprocals and the final scaling by 1/r_ii are not
 * counted there, as the paper counts only the n^3 terms.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

typedef struct { double re, im; } zc;

static inline zc z_make(double re, double im) { zc r; r.re = re; r.im = im; return r; }
static inline zc z_mul(zc a, zc b) { return z_make(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re); }
static inline zc z_conj(zc a) { return z_make(a.re, -a.im); }
static inline zc z_add(zc a, zc b) { return z_make(a.re + b.re, a.im + b.im); }
static inline zc z_sub(zc a, zc b) { return z_make(a.re - b.re, a.im - b.im); }
static inline zc z_divr(zc a, double d) { return z_make(a.re / d, a.im / d); }

#define CNT(m) do { if (m) ++*(m); } while (0)

/* ------------------------------------------------------------------------- */
/* Cholesky, Eqs. 3-4: row i of R from rows 1..i-1.                          */
/* Returns 0, or the 1-based row whose pivot argument is <= 0 or not finite. */
/* R's strictly lower part is written as zero.  R may not alias A.           */
/* ------------------------------------------------------------------------- */
int orc_chol_d(int n, const double* A, double* R, long long* mults)
{
    memset(R, 0, sizeof(double) * (size_t)n * n);
    for (int i = 0; i < n; ++i) {
        /* Eq. 3: r_ii = sqrt(a_ii - sum_{k<i} r_ki^* r_ki) */
        double t = A[i * n + i];
        for (int k = 0; k < i; ++k) { t -= R[k * n + i] * R[k * n + i]; CNT(mults); }
        if (!(t > 0.0) || !isfinite(t)) return i + 1;
        double rii = sqrt(t);
        R[i * n + i] = rii;
        /* Eq. 4: r_ij = (a_ij - sum_{k<i} r_ki^* r_kj) / r_ii, j > i */
        for (int j = i + 1; j < n; ++j) {
            double s = A[i * n + j];
            for (int k = 0; k < i; ++k) { s -= R[k * n + i] * R[k * n + j]; CNT(mults); }
            R[i * n + j] = s / rii;
        }
    }
    return 0;
}

int orc_chol_z(int n, const double* Ad, double* Rd, long long* mults)
{
    const zc* A = (const zc*)Ad;
    zc* R = (zc*)Rd;
    memset(R, 0, sizeof(zc) * (size_t)n * n);
    for (int i = 0; i < n; ++i) {
        /* Eq. 3 with r_ki^* r_ki = |r_ki|^2, a real number */
        double t = A[i * n + i].re;
        for (int k = 0; k < i; ++k) {
            zc p = z_mul(z_conj(R[k * n + i]), R[k * n + i]);
            t -= p.re;
            CNT(mults);
        }
        if (!(t > 0.0) || !isfinite(t)) return i + 1;
        double rii = sqrt(t);
        R[i * n + i] = z_make(rii, 0.0);
        /* Eq. 4, conjugate on the first factor */
        for (int j = i + 1; j < n; ++j) {
            zc s = A[i * n + j];
            for (int k = 0; k < i; ++k) { s = z_sub(s, z_mul(z_conj(R[k * n + i]), R[k * n + j])); CNT(mults); }
            R[i * n + j] = z_divr(s, rii);
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Proposed inverse, Eqs. 20-24: solve R X = S with s_ij = delta_ij / r_ii   */
/* (S is the upper part of B = R^{-*}), upper half x_ij, i <= j only; an     */
/* entry below the diagonal is taken as the conjugate of its mirror.         */
/*   x_ij = (s_ij - sum_{k>i} r_ik x~_kj) / r_ii,                            */
/*   x~_kj = x_kj (k <= j), conj(x_jk) (k > j).                              */
/* Row order: i = N..1; within a row j = N..i+1, then the diagonal.          */
/* X's strictly lower part is written as zero.                               */
/* ------------------------------------------------------------------------- */
void orc_inv_rows_d(int n, const double* R, double* X, long long* mults)
{
    memset(X, 0, sizeof(double) * (size_t)n * n);
    for (int i = n - 1; i >= 0; --i) {
        double rii = R[i * n + i];
        for (int j = n - 1; j > i; --j) {
            double s = 0.0;
            for (int k = i + 1; k < n; ++k) {
                double xt = (k <= j) ? X[k * n + j] : X[j * n + k];
                s += R[i * n + k] * xt;
                CNT(mults);
            }
            X[i * n + j] = (0.0 - s) / rii;
        }
        double s = 0.0;
        for (int k = i + 1; k < n; ++k) { s += R[i * n + k] * X[i * n + k]; CNT(mults); }
        X[i * n + i] = (1.0 / rii - s) / rii;
    }
}

void orc_inv_rows_z(int n, const double* Rd, double* Xd, long long* mults)
{
    const zc* R = (const zc*)Rd;
    zc* X = (zc*)Xd;
    memset(X, 0, sizeof(zc) * (size_t)n * n);
    for (int i = n - 1; i >= 0; --i) {
        double rii = R[i * n + i].re;
        for (int j = n - 1; j > i; --j) {
            zc s = z_make(0.0, 0.0);
            for (int k = i + 1; k < n; ++k) {
                zc xt = (k <= j) ? X[k * n + j] : z_conj(X[j * n + k]);
                s = z_add(s, z_mul(R[i * n + k], xt));
                CNT(mults);
            }
            X[i * n + j] = z_divr(z_sub(z_make(0.0, 0.0), s), rii);
        }
        zc s = z_make(0.0, 0.0);
        for (int k = i + 1; k < n; ++k) { s = z_add(s, z_mul(R[i * n + k], z_conj(X[i * n + k]))); CNT(mults); }
        /* the diagonal of a Hermitian inverse is real: keep the real part */
        X[i * n + i] = z_make((1.0 / rii - s.re) / rii, 0.0);
    }
}

/* Same solve taken column by column ("R x_i = s_i"): j = N..1, i = j..1. */
void orc_inv_cols_d(int n, const double* R, double* X, long long* mults)
{
    memset(X, 0, sizeof(double) * (size_t)n * n);
    for (int j = n - 1; j >= 0; --j) {
        for (int i = j; i >= 0; --i) {
            double rii = R[i * n + i];
            double s = 0.0;
            for (int k = i + 1; k < n; ++k) {
                double xt = (k <= j) ? X[k * n + j] : X[j * n + k];
                s += R[i * n + k] * xt;
                CNT(mults);
            }
            double sij = (i == j) ? 1.0 / rii : 0.0;
            X[i * n + j] = (sij - s) / rii;
        }
    }
}

void orc_inv_cols_z(int n, const double* Rd, double* Xd, long long* mults)
{
    const zc* R = (const zc*)Rd;
    zc* X = (zc*)Xd;
    memset(X, 0, sizeof(zc) * (size_t)n * n);
    for (int j = n - 1; j >= 0; --j) {
        for (int i = j; i >= 0; --i) {
            double rii = R[i * n + i].re;
            zc s = z_make(0.0, 0.0);
            for (int k = i + 1; k < n; ++k) {
                zc xt = (k <= j) ? X[k * n + j] : z_conj(X[j * n + k]);
                s = z_add(s, z_mul(R[i * n + k], xt));
                CNT(mults);
            }
            if (i == j) X[i * n + j] = z_make((1.0 / rii - s.re) / rii, 0.0);
            else        X[i * n + j] = z_divr(z_sub(z_make(0.0, 0.0), s), rii);
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Existing method A, "Equation Solving" (Eq. 15): for each column j solve   */
/* R^* b = e_j (forward) then R x_j = b (backward), upper half only, with    */
/* x~ as above.  Counting follows the paper's accounting: the unknowns of    */
/* each solve are restricted to the triangle (b_k, k >= j; x_ij, i <= j) but */
/* every dot product runs over its full remaining index range.               */
/* ------------------------------------------------------------------------- */
void orc_es_d(int n, const double* R, double* X, long long* mults)
{
    double* b = (double*)calloc((size_t)n, sizeof(double));
    memset(X, 0, sizeof(double) * (size_t)n * n);
    for (int j = n - 1; j >= 0; --j) {
        for (int k = 0; k < n; ++k) b[k] = 0.0;
        for (int k = j; k < n; ++k) {           /* forward: L = R^*, l_kl = conj(r_lk) */
            double s = (k == j) ? 1.0 : 0.0;
            for (int l = 0; l < k; ++l) { s -= R[l * n + k] * b[l]; CNT(mults); }
            b[k] = s / R[k * n + k];
        }
        for (int i = j; i >= 0; --i) {          /* backward, rows i <= j */
            double s = 0.0;
            for (int l = i + 1; l < n; ++l) {
                double xt = (l <= j) ? X[l * n + j] : X[j * n + l];
                s += R[i * n + l] * xt;
                CNT(mults);
            }
            X[i * n + j] = (b[i] - s) / R[i * n + i];
        }
    }
    free(b);
}

void orc_es_z(int n, const double* Rd, double* Xd, long long* mults)
{
    const zc* R = (const zc*)Rd;
    zc* X = (zc*)Xd;
    zc* b = (zc*)calloc((size_t)n, sizeof(zc));
    memset(X, 0, sizeof(zc) * (size_t)n * n);
    for (int j = n - 1; j >= 0; --j) {
        for (int k = 0; k < n; ++k) b[k] = z_make(0.0, 0.0);
        for (int k = j; k < n; ++k) {
            zc s = z_make((k == j) ? 1.0 : 0.0, 0.0);
            for (int l = 0; l < k; ++l) { s = z_sub(s, z_mul(z_conj(R[l * n + k]), b[l])); CNT(mults); }
            b[k] = z_divr(s, R[k * n + k].re);
        }
        for (int i = j; i >= 0; --i) {
            zc s = z_make(0.0, 0.0);
            for (int l = i + 1; l < n; ++l) {
                zc xt = (l <= j) ? X[l * n + j] : z_conj(X[j * n + l]);
                s = z_add(s, z_mul(R[i * n + l], xt));
                CNT(mults);
            }
            s = z_sub(b[i], s);
            if (i == j) X[i * n + j] = z_make(s.re / R[i * n + i].re, 0.0);
            else        X[i * n + j] = z_divr(s, R[i * n + i].re);
        }
    }
    free(b);
}

/* ------------------------------------------------------------------------- */
/* Existing method B, "Triangular Matrix Operations" (Eqs. 16-19):          */
/* M = R^{-1} column by column from R m_i = e_i (Eq. 18), then X = M M^*     */
/* (Eq. 19), upper half.  exploit = 0: the paper's accounting (the dots of   */
/* the triangular solve run over k+1..N); exploit = 1: dots stop at the last */
/* nonzero of m_i (the structure-exploiting count, LAPACK TRTRI style).      */
/* ------------------------------------------------------------------------- */
void orc_tmo_d(int n, const double* R, double* X, int exploit, long long* mults)
{
    double* M = (double*)calloc((size_t)n * n, sizeof(double));
    for (int i = 0; i < n; ++i) {
        for (int k = i; k >= 0; --k) {
            double s = (k == i) ? 1.0 : 0.0;
            int lend = exploit ? i + 1 : n;
            for (int l = k + 1; l < lend; ++l) { s -= R[k * n + l] * M[l * n + i]; CNT(mults); }
            M[k * n + i] = s / R[k * n + k];
        }
    }
    memset(X, 0, sizeof(double) * (size_t)n * n);
    for (int i = 0; i < n; ++i)
        for (int j = i; j < n; ++j) {
            double s = 0.0;
            for (int l = j; l < n; ++l) { s += M[i * n + l] * M[j * n + l]; CNT(mults); }
            X[i * n + j] = s;
        }
    free(M);
}

void orc_tmo_z(int n, const double* Rd, double* Xd, int exploit, long long* mults)
{
    const zc* R = (const zc*)Rd;
    zc* X = (zc*)Xd;
    zc* M = (zc*)calloc((size_t)n * n, sizeof(zc));
    for (int i = 0; i < n; ++i) {
        for (int k = i; k >= 0; --k) {
            zc s = z_make((k == i) ? 1.0 : 0.0, 0.0);
            int lend = exploit ? i + 1 : n;
            for (int l = k + 1; l < lend; ++l) { s = z_sub(s, z_mul(R[k * n + l], M[l * n + i])); CNT(mults); }
            M[k * n + i] = z_divr(s, R[k * n + k].re);
        }
    }
    memset(X, 0, sizeof(zc) * (size_t)n * n);
    for (int i = 0; i < n; ++i)
        for (int j = i; j < n; ++j) {
            zc s = z_make(0.0, 0.0);
            for (int l = j; l < n; ++l) { s = z_add(s, z_mul(M[i * n + l], z_conj(M[j * n + l]))); CNT(mults); }
            if (i == j) s.im = 0.0;
            X[i * n + j] = s;
        }
    free(M);
}

/* ------------------------------------------------------------------------- */
/* LDL, Eqs. 10-11: A = R^* D R with unit upper R.                           */
/*   d_i  = a_ii - sum_{k<i} r_ki^* r_ki d_k                                 */
/*   r_ij = (a_ij - sum_{k<i} r_ki^* r_kj d_k) / d_i                         */
/* The products are formed left to right: (r_ki^* r_kj) d_k.                 */
/* R gets ones on its diagonal; d receives D.  Returns info like Cholesky    */
/* (a pivot d_i <= 0 or not finite).                                         */
/* ------------------------------------------------------------------------- */
int orc_ldl_d(int n, const double* A, double* R, double* d, long long* mults)
{
    memset(R, 0, sizeof(double) * (size_t)n * n);
    for (int i = 0; i < n; ++i) {
        double t = A[i * n + i];
        for (int k = 0; k < i; ++k) { t -= R[k * n + i] * R[k * n + i] * d[k]; CNT(mults); }
        if (!(t > 0.0) || !isfinite(t)) return i + 1;
        d[i] = t;
        R[i * n + i] = 1.0;
        for (int j = i + 1; j < n; ++j) {
            double s = A[i * n + j];
            for (int k = 0; k < i; ++k) { s -= R[k * n + i] * R[k * n + j] * d[k]; CNT(mults); }
            R[i * n + j] = s / t;
        }
    }
    return 0;
}

int orc_ldl_z(int n, const double* Ad, double* Rd, double* d, long long* mults)
{
    const zc* A = (const zc*)Ad;
    zc* R = (zc*)Rd;
    memset(R, 0, sizeof(zc) * (size_t)n * n);
    for (int i = 0; i < n; ++i) {
        double t = A[i * n + i].re;
        for (int k = 0; k < i; ++k) {
            zc p = z_mul(z_conj(R[k * n + i]), R[k * n + i]);
            t -= p.re * d[k];
            CNT(mults);
        }
        if (!(t > 0.0) || !isfinite(t)) return i + 1;
        d[i] = t;
        R[i * n + i] = z_make(1.0, 0.0);
        for (int j = i + 1; j < n; ++j) {
            zc s = A[i * n + j];
            for (int k = 0; k < i; ++k) {
                zc p = z_mul(z_conj(R[k * n + i]), R[k * n + j]);
                s = z_sub(s, z_make(p.re * d[k], p.im * d[k]));
                CNT(mults);
            }
            R[i * n + j] = z_divr(s, t);
        }
    }
    return 0;
}

/* Proposed inverse via LDL, Eqs. 25-29: R X = S~ with s~_ij = delta_ij/d_i, */
/* R unit upper, so x_ij = s~_ij - sum_{k>i} r_ik x~_kj.  Rows N..1.         */
void orc_ldl_inv_d(int n, const double* R, const double* d, double* X, long long* mults)
{
    memset(X, 0, sizeof(double) * (size_t)n * n);
    for (int i = n - 1; i >= 0; --i) {
        for (int j = n - 1; j > i; --j) {
            double s = 0.0;
            for (int k = i + 1; k < n; ++k) {
                double xt = (k <= j) ? X[k * n + j] : X[j * n + k];
                s += R[i * n + k] * xt;
                CNT(mults);
            }
            X[i * n + j] = 0.0 - s;
        }
        double s = 0.0;
        for (int k = i + 1; k < n; ++k) { s += R[i * n + k] * X[i * n + k]; CNT(mults); }
        X[i * n + i] = 1.0 / d[i] - s;
    }
}

void orc_ldl_inv_z(int n, const double* Rd, const double* d, double* Xd, long long* mults)
{
    const zc* R = (const zc*)Rd;
    zc* X = (zc*)Xd;
    memset(X, 0, sizeof(zc) * (size_t)n * n);
    for (int i = n - 1; i >= 0; --i) {
        for (int j = n - 1; j > i; --j) {
            zc s = z_make(0.0, 0.0);
            for (int k = i + 1; k < n; ++k) {
                zc xt = (k <= j) ? X[k * n + j] : z_conj(X[j * n + k]);
                s = z_add(s, z_mul(R[i * n + k], xt));
                CNT(mults);
            }
            X[i * n + j] = z_sub(z_make(0.0, 0.0), s);
        }
        zc s = z_make(0.0, 0.0);
        for (int k = i + 1; k < n; ++k) { s = z_add(s, z_mul(R[i * n + k], z_conj(X[i * n + k]))); CNT(mults); }
        X[i * n + i] = z_make(1.0 / d[i] - s.re, 0.0);
    }
}

/* ------------------------------------------------------------------------- */
/* Gauss-Jordan elimination with partial pivoting in long double on the full */
/* matrix [A | I] (A symmetrised from its upper triangle).  An independent   */
/* inverse used only to check the routines above.  Returns 0, or 1 if a      */
/* pivot is exactly zero.  X receives the full inverse rounded to double.    */
/* ------------------------------------------------------------------------- */
int orc_gj_ld(int n, const double* A, double* X)
{
    long double* W = (long double*)calloc((size_t)n * 2 * n, sizeof(long double));
    int w = 2 * n, rc = 0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            W[i * w + j] = (long double)(i <= j ? A[i * n + j] : A[j * n + i]);
            W[i * w + n + j] = (i == j) ? 1.0L : 0.0L;
        }
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r) if (fabsl(W[r * w + c]) > fabsl(W[p * w + c])) p = r;
        if (W[p * w + c] == 0.0L) { rc = 1; break; }
        if (p != c) for (int j = 0; j < w; ++j) { long double t = W[c * w + j]; W[c * w + j] = W[p * w + j]; W[p * w + j] = t; }
        long double piv = W[c * w + c];
        for (int j = 0; j < w; ++j) W[c * w + j] /= piv;
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            long double f = W[r * w + c];
            if (f == 0.0L) continue;
            for (int j = 0; j < w; ++j) W[r * w + j] -= f * W[c * w + j];
        }
    }
    for (int i = 0; i < n; ++i) for (int j = 0; j < n; ++j) X[i * n + j] = (double)W[i * w + n + j];
    free(W);
    return rc;
}

typedef struct { long double re, im; } lzc;
static inline lzc lz_mul(lzc a, lzc b) { lzc r; r.re = a.re * b.re - a.im * b.im; r.im = a.re * b.im + a.im * b.re; return r; }
static inline long double lz_abs2(lzc a) { return a.re * a.re + a.im * a.im; }

int orc_gj_lz(int n, const double* Ad, double* Xd)
{
    const zc* A = (const zc*)Ad;
    zc* X = (zc*)Xd;
    int w = 2 * n, rc = 0;
    lzc* W = (lzc*)calloc((size_t)n * w, sizeof(lzc));
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            zc a = (i <= j) ? A[i * n + j] : z_conj(A[j * n + i]);
            if (i == j) a.im = 0.0;
            W[i * w + j].re = a.re; W[i * w + j].im = a.im;
            W[i * w + n + j].re = (i == j) ? 1.0L : 0.0L; W[i * w + n + j].im = 0.0L;
        }
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r) if (lz_abs2(W[r * w + c]) > lz_abs2(W[p * w + c])) p = r;
        long double m2 = lz_abs2(W[p * w + c]);
        if (m2 == 0.0L) { rc = 1; break; }
        if (p != c) for (int j = 0; j < w; ++j) { lzc t = W[c * w + j]; W[c * w + j] = W[p * w + j]; W[p * w + j] = t; }
        lzc piv = W[c * w + c];
        lzc inv; inv.re = piv.re / m2; inv.im = -piv.im / m2;
        for (int j = 0; j < w; ++j) W[c * w + j] = lz_mul(W[c * w + j], inv);
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            lzc f = W[r * w + c];
            if (f.re == 0.0L && f.im == 0.0L) continue;
            for (int j = 0; j < w; ++j) {
                lzc t = lz_mul(f, W[c * w + j]);
                W[r * w + j].re -= t.re; W[r * w + j].im -= t.im;
            }
        }
    }
    for (int i = 0; i < n; ++i) for (int j = 0; j < n; ++j) { X[i * n + j].re = (double)W[i * w + n + j].re; X[i * n + j].im = (double)W[i * w + n + j].im; }
    free(W);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Adjoint of X = A^{-1} on the Hermitian subspace:                           */
/*   dA = -X S X,  S = (G + G^H)/2,                                          */
/* with X the full Hermitian inverse and G the full gradient of the loss     */
/* with respect to X.  Plain triple loops, T = S X first, then dA = -X T.    */
/* ------------------------------------------------------------------------- */
void orc_grad_d(int n, const double* X, const double* G, double* dA)
{
    double* S = (double*)malloc(sizeof(double) * (size_t)n * n);
    double* T = (double*)malloc(sizeof(double) * (size_t)n * n);
    for (int i = 0; i < n; ++i) for (int j = 0; j < n; ++j) S[i * n + j] = 0.5 * (G[i * n + j] + G[j * n + i]);
    for (int i = 0; i < n; ++i) for (int j = 0; j < n; ++j) {
        double s = 0.0;
        for (int k = 0; k < n; ++k) s += S[i * n + k] * X[k * n + j];
        T[i * n + j] = s;
    }
    for (int i = 0; i < n; ++i) for (int j = 0; j < n; ++j) {
        double s = 0.0;
        for (int k = 0; k < n; ++k) s += X[i * n + k] * T[k * n + j];
        dA[i * n + j] = -s;
    }
    free(S); free(T);
}

void orc_grad_z(int n, const double* Xd, const double* Gd, double* dAd)
{
    const zc* X = (const zc*)Xd;
    const zc* G = (const zc*)Gd;
    zc* dA = (zc*)dAd;
    zc* S = (zc*)malloc(sizeof(zc) * (size_t)n * n);
    zc* T = (zc*)malloc(sizeof(zc) * (size_t)n * n);
    for (int i = 0; i < n; ++i) for (int j = 0; j < n; ++j) {
        zc g = z_add(G[i * n + j], z_conj(G[j * n + i]));
        S[i * n + j] = z_make(0.5 * g.re, 0.5 * g.im);
    }
    for (int i = 0; i < n; ++i) for (int j = 0; j < n; ++j) {
        zc s = z_make(0.0, 0.0);
        for (int k = 0; k < n; ++k) s = z_add(s, z_mul(S[i * n + k], X[k * n + j]));
        T[i * n + j] = s;
    }
    for (int i = 0; i < n; ++i) for (int j = 0; j < n; ++j) {
        zc s = z_make(0.0, 0.0);
        for (int k = 0; k < n; ++k) s = z_add(s, z_mul(X[i * n + k], T[k * n + j]));
        dA[i * n + j] = z_make(-s.re, -s.im);
    }
    free(S); free(T);
}

/* ------------------------------------------------------------------------- */
/* Batched driver.  Matrix b has order n[b] and starts at element off[b] of  */
/* A, R and X (layout 0: dense row-major n*n; layout 1: upper triangle       */
/* packed row by row, n(n+1)/2 elements).  cplx selects complex128 (pairs of */
/* doubles).  R may be NULL.  X receives the upper half (dense: the lower    */
/* part of X is left as it was unless fill_lower, which writes the conjugate */
/* mirror).  info[b] = 0 or the failing 1-based row (then R and X of that    */
/* matrix are left untouched).  Matrices are split over nthreads threads.    */
/* ------------------------------------------------------------------------- */
typedef struct {
    int cplx, layout, fill_lower, maxn;
    const int* n; const long long* off;
    const double* A; double* R; double* X; int* info;
    long long b0, b1;
} orc_job;

static void orc_unpack(int n, int layout, int c, const double* src, double* dst)
{
    for (int i = 0; i < n; ++i)
        for (int j = i; j < n; ++j) {
            size_t s = layout ? (size_t)i * n - (size_t)i * (i - 1) / 2 + (size_t)(j - i) : (size_t)i * n + j;
            for (int q = 0; q < c; ++q) dst[((size_t)i * n + j) * c + q] = src[s * c + q];
        }
}

static void orc_pack(int n, int layout, int c, int fill_lower, const double* src, double* dst)
{
    for (int i = 0; i < n; ++i)
        for (int j = i; j < n; ++j) {
            size_t s = layout ? (size_t)i * n - (size_t)i * (i - 1) / 2 + (size_t)(j - i) : (size_t)i * n + j;
            for (int q = 0; q < c; ++q) dst[s * c + q] = src[((size_t)i * n + j) * c + q];
            if (!layout && fill_lower && j > i) {
                size_t m = (size_t)j * n + i;
                dst[m * c] = src[((size_t)i * n + j) * c];
                if (c == 2) dst[m * c + 1] = -src[((size_t)i * n + j) * c + 1];
            }
        }
}

static void* orc_worker(void* p)
{
    orc_job* jb = (orc_job*)p;
    int c = jb->cplx ? 2 : 1;
    size_t sz = (size_t)jb->maxn * jb->maxn * c;
    double* a = (double*)calloc(sz, sizeof(double));
    double* r = (double*)calloc(sz, sizeof(double));
    double* x = (double*)calloc(sz, sizeof(double));
    for (long long b = jb->b0; b < jb->b1; ++b) {
        int n = jb->n[b];
        size_t o = (size_t)jb->off[b] * c;
        if (n <= 0) { jb->info[b] = 0; continue; }
        memset(a, 0, sizeof(double) * (size_t)n * n * c);
        orc_unpack(n, jb->layout, c, jb->A + o, a);
        int info = jb->cplx ? orc_chol_z(n, a, r, NULL) : orc_chol_d(n, a, r, NULL);
        jb->info[b] = info;
        if (info) continue;
        if (jb->cplx) orc_inv_rows_z(n, r, x, NULL); else orc_inv_rows_d(n, r, x, NULL);
        if (jb->R) orc_pack(n, jb->layout, c, 0, r, jb->R + o);
        orc_pack(n, jb->layout, c, jb->fill_lower, x, jb->X + o);
        if (jb->R && !jb->layout)            /* dense R: strictly lower part is zero */
            for (int i = 1; i < n; ++i) for (int j = 0; j < i; ++j) for (int q = 0; q < c; ++q)
                jb->R[o + ((size_t)i * n + j) * c + q] = 0.0;
    }
    free(a); free(r); free(x);
    return NULL;
}

int orc_inv_batch(int cplx, long long batch, const int* n, const long long* off, int layout, int fill_lower,
                  const double* A, double* R, double* X, int* info, int nthreads)
{
    if (batch <= 0) return 0;
    int maxn = 1;
    for (long long b = 0; b < batch; ++b) if (n[b] > maxn) maxn = n[b];
    if (nthreads < 1) nthreads = 1;
    if (nthreads > batch) nthreads = (int)batch;
    orc_job* jobs = (orc_job*)calloc((size_t)nthreads, sizeof(orc_job));
    pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
    for (int t = 0; t < nthreads; ++t) {
        orc_job j = { cplx, layout, fill_lower, maxn, n, off, A, R, X, info,
                      batch * t / nthreads, batch * (t + 1) / nthreads };
        jobs[t] = j;
    }
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, orc_worker, &jobs[t]);
    orc_worker(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(jobs); free(th);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Large single matrices (threads).  orc_chol_mt_d and orc_inv_rows_mt_d     */
/* perform exactly the operations of orc_chol_d and orc_inv_rows_d, with the */
/* same operands in the same order for every entry (so the results are the  */
/* same bits); only the entries of one row are shared out over threads, and */
/* a transposed copy keeps each inner sum on contiguous memory.              */
/* ------------------------------------------------------------------------- */
typedef struct {
    int n, t, nt;
    const double* A; double* R; double* L;   /* L[j*n+k] = r_kj (k <= j) */
    double* X; double* F;                    /* F: full symmetric X (F[j*n+k] = x~_kj) */
    double* piv; int* info;
    pthread_barrier_t* bar;
} orc_mt;

static void* orc_chol_mt_worker(void* p)
{
    orc_mt* w = (orc_mt*)p;
    const int n = w->n;
    double* L = w->L;
    for (int i = 0; i < n; ++i) {
        if (w->t == 0) {
            /* Eq. 3 */
            double t = w->A[(size_t)i * n + i];
            for (int k = 0; k < i; ++k) t -= L[(size_t)i * n + k] * L[(size_t)i * n + k];
            if (!(t > 0.0) || !isfinite(t)) { if (*w->info == 0) *w->info = i + 1; }
            *w->piv = sqrt(t);
            L[(size_t)i * n + i] = *w->piv;
        }
        pthread_barrier_wait(w->bar);
        if (*w->info) return NULL;
        const double rii = *w->piv;
        /* Eq. 4 for j = i+1..n-1, this thread's share */
        for (int j = i + 1 + w->t; j < n; j += w->nt) {
            double s = w->A[(size_t)i * n + j];
            for (int k = 0; k < i; ++k) s -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
            L[(size_t)j * n + i] = s / rii;
        }
        pthread_barrier_wait(w->bar);
    }
    return NULL;
}

static void orc_run_mt(orc_mt* base, int nthreads, void* (*fn)(void*))
{
    pthread_barrier_t bar;
    pthread_barrier_init(&bar, NULL, (unsigned)nthreads);
    orc_mt* jobs = (orc_mt*)calloc((size_t)nthreads, sizeof(orc_mt));
    pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
    for (int t = 0; t < nthreads; ++t) { jobs[t] = *base; jobs[t].t = t; jobs[t].nt = nthreads; jobs[t].bar = &bar; }
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, fn, &jobs[t]);
    fn(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
    pthread_barrier_destroy(&bar);
    free(jobs); free(th);
}

/* Cholesky (Eqs. 3-4) as orc_chol_d; returns 0 or the failing 1-based row. */
int orc_chol_mt_d(int n, const double* A, double* R, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    double* L = (double*)calloc((size_t)n * n, sizeof(double));
    double piv = 0.0;
    int info = 0;
    orc_mt base = { n, 0, 1, A, R, L, NULL, NULL, &piv, &info, NULL };
    orc_run_mt(&base, nthreads, orc_chol_mt_worker);
    memset(R, 0, sizeof(double) * (size_t)n * n);
    if (info == 0)
        for (int j = 0; j < n; ++j)
            for (int k = 0; k <= j; ++k) R[(size_t)k * n + j] = L[(size_t)j * n + k];
    free(L);
    return info;
}

static void* orc_inv_mt_worker(void* p)
{
    orc_mt* w = (orc_mt*)p;
    const int n = w->n;
    const double* R = w->R;
    double* F = w->F;
    for (int i = n - 1; i >= 0; --i) {
        const double rii = R[(size_t)i * n + i];
        /* x_ij, j = i+1..n-1 (Sec. IV.A); F's row j holds x~_kj for every k > i */
        for (int j = i + 1 + w->t; j < n; j += w->nt) {
            double s = 0.0;
            for (int k = i + 1; k < n; ++k) s += R[(size_t)i * n + k] * F[(size_t)j * n + k];
            const double x = (0.0 - s) / rii;
            F[(size_t)i * n + j] = x;
            F[(size_t)j * n + i] = x;
        }
        pthread_barrier_wait(w->bar);
        if (w->t == 0) {
            double s = 0.0;
            for (int k = i + 1; k < n; ++k) s += R[(size_t)i * n + k] * F[(size_t)i * n + k];
            F[(size_t)i * n + i] = (1.0 / rii - s) / rii;
        }
        pthread_barrier_wait(w->bar);
    }
    return NULL;
}

/* Proposed inverse (Sec. IV.A) as orc_inv_rows_d: upper half of X, lower zero. */
void orc_inv_rows_mt_d(int n, const double* R, double* X, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    double* F = (double*)calloc((size_t)n * n, sizeof(double));
    orc_mt base = { n, 0, 1, NULL, (double*)R, NULL, NULL, F, NULL, NULL, NULL };
    orc_run_mt(&base, nthreads, orc_inv_mt_worker);
    memset(X, 0, sizeof(double) * (size_t)n * n);
    for (int i = 0; i < n; ++i)
        for (int j = i; j < n; ++j) X[(size_t)i * n + j] = F[(size_t)i * n + j];
    free(F);
}

/* Columns cols[0..ncols-1] of A^{-1} = R^{-1} R^{-*}, each from the two      */
/* triangular solves of Eq. 15 for the right-hand side e_j: the forward     */
/* solve R^* y = e_j (y_k = 0 for k < j; each y_k's terms in ascending l,    */
/* taken column by column over R's rows), then the back solve R x = y over  */
/* every row.  Xc[c*n + i] = (A^{-1})_{i, cols[c]}.  Threads over columns.   */
typedef struct { int n, ncols, t, nt; const double* R; const int* cols; double* Xc; } orc_cols_job;

static void* orc_cols_worker(void* p)
{
    orc_cols_job* w = (orc_cols_job*)p;
    const int n = w->n;
    const double* R = w->R;
    double* y = (double*)calloc((size_t)n, sizeof(double));
    for (int c = w->t; c < w->ncols; c += w->nt) {
        const int j = w->cols[c];
        double* x = w->Xc + (size_t)c * n;
        /* forward: y_k = (delta_kj - sum_{l<k} r_lk y_l) / r_kk */
        for (int k = 0; k < n; ++k) y[k] = (k == j) ? 1.0 : 0.0;
        for (int l = j; l < n; ++l) {
            y[l] = y[l] / R[(size_t)l * n + l];
            for (int k = l + 1; k < n; ++k) y[k] -= R[(size_t)l * n + k] * y[l];
        }
        /* back: x_i = (y_i - sum_{l>i} r_il x_l) / r_ii, i = n-1..0 */
        for (int i = n - 1; i >= 0; --i) {
            double s = 0.0;
            for (int l = i + 1; l < n; ++l) s += R[(size_t)i * n + l] * x[l];
            x[i] = (y[i] - s) / R[(size_t)i * n + i];
        }
    }
    free(y);
    return NULL;
}

void orc_solve_cols_d(int n, const double* R, int ncols, const int* cols, double* Xc, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > ncols) nthreads = ncols > 0 ? ncols : 1;
    orc_cols_job* jobs = (orc_cols_job*)calloc((size_t)nthreads, sizeof(orc_cols_job));
    pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
    for (int t = 0; t < nthreads; ++t) {
        orc_cols_job j = { n, ncols, t, nthreads, R, cols, Xc };
        jobs[t] = j;
    }
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, orc_cols_worker, &jobs[t]);
    orc_cols_worker(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(jobs); free(th);
}
