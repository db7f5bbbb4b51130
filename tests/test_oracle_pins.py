"""Pins for the CPU oracle: facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself.  Each test checks it against a
closed form, a special case, an invariant, an independent method (Gauss-Jordan
in long double, finite differences) or the operation counts the paper prints
(Table 1).  A dropped term, a wrong sign or index, or a conjugate on the wrong
factor in Eqs. 3-4 or in the Sec. IV.A recurrence fails at least one of them.
"""
import json
import os
from fractions import Fraction
from math import comb

import numpy as np
import pytest

from paper_1111_4144_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rand_hpd(rng, n, cplx, shift=None):
    if cplx:
        B = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    else:
        B = rng.standard_normal((n, n))
    A = B @ np.conj(B).T + (n if shift is None else shift) * np.eye(n)
    return 0.5 * (A + np.conj(A).T)


def full(Xu):
    return np.triu(Xu) + np.conj(np.triu(Xu, 1)).T


# --------------------------------------------------------------------------
# closed forms
# --------------------------------------------------------------------------
@pytest.mark.parametrize("cplx", [False, True])
def test_2x2_closed_form(orc, cplx):
    """[[a,b],[b*,c]]: r11=sqrt(a), r12=b/sqrt(a), r22=sqrt(c-|b|^2/a); X = adj/det."""
    a, c = 2.5, 1.75
    b = (0.6 - 0.45j) if cplx else 0.6
    A = np.array([[a, b], [np.conj(b), c]])
    R, info = orc.chol(A)
    assert info == 0
    det = a * c - abs(b) ** 2
    Rx = np.array([[np.sqrt(a), b / np.sqrt(a)], [0, np.sqrt(c - abs(b) ** 2 / a)]])
    Xx = np.array([[c, -b], [-np.conj(b), a]]) / det
    np.testing.assert_allclose(R, Rx, rtol=1e-15, atol=1e-15)
    X = orc.inv_rows(R)
    np.testing.assert_allclose(X, np.triu(Xx), rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("n", [1, 2, 5, 17])
def test_diagonal_and_identity(orc, n):
    d = np.linspace(0.5, 9.0, n)
    R, info = orc.chol(np.diag(d))
    assert info == 0
    np.testing.assert_allclose(R, np.diag(np.sqrt(d)), rtol=1e-15)
    np.testing.assert_allclose(orc.inv_rows(R), np.diag(1.0 / d), rtol=1e-15)
    R, _ = orc.chol(np.eye(n))
    assert np.array_equal(R, np.eye(n)) and np.array_equal(orc.inv_rows(R), np.eye(n))


@pytest.mark.parametrize("n", [1, 3, 8, 16, 33])
@pytest.mark.parametrize("cplx", [False, True])
def test_min_matrix_exact(orc, n, cplx):
    """a_ij = min(i,j): R = all-ones upper triangle; A^-1 = tridiag(-1,2,-1) with x_NN = 1."""
    i = np.arange(1, n + 1)
    A = np.minimum.outer(i, i).astype(np.complex128 if cplx else np.float64)
    R, info = orc.chol(A)
    assert info == 0
    assert np.array_equal(R, np.triu(np.ones((n, n))))
    X = orc.inv_rows(R)
    T = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    T[-1, -1] = 1
    assert np.array_equal(X, np.triu(T))
    assert np.array_equal(orc.inv_cols(R), np.triu(T))


@pytest.mark.parametrize("n", [2, 6, 13, 32])
def test_tridiagonal_closed_form(orc, n):
    """T = tridiag(-1,2,-1): r_ii = sqrt((i+1)/i), r_i,i+1 = -sqrt(i/(i+1)); (T^-1)_ij = i(N+1-j)/(N+1)."""
    T = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    R, info = orc.chol(T)
    assert info == 0
    i = np.arange(1, n + 1, dtype=float)
    Rx = np.diag(np.sqrt((i + 1) / i)) + np.diag(-np.sqrt(i[:-1] / (i[:-1] + 1)), 1)
    np.testing.assert_allclose(R, Rx, rtol=1e-14, atol=1e-15)
    X = orc.inv_rows(R)
    I, J = np.meshgrid(i, i, indexing="ij")
    Xx = np.triu(I * (n + 1 - J) / (n + 1))
    np.testing.assert_allclose(X, Xx, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("n", [1, 4, 8, 10])
def test_pascal_exact_integers(orc, n):
    """Symmetric Pascal P_ij = C(i+j, i): R_ij = C(j, i); P^-1 = L^-T L^-1, L^-1_ij = (-1)^(i-j) C(i,j)."""
    P = np.array([[comb(i + j, i) for j in range(n)] for i in range(n)], dtype=np.float64)
    R, info = orc.chol(P)
    assert info == 0
    Rx = np.array([[comb(j, i) for j in range(n)] for i in range(n)], dtype=np.float64)
    assert np.array_equal(R, Rx)
    Li = [[(-1) ** (i - j) * comb(i, j) if j <= i else 0 for j in range(n)] for i in range(n)]
    Pinv = [[sum(Li[k][i] * Li[k][j] for k in range(n)) for j in range(n)] for i in range(n)]
    X = orc.inv_rows(R)
    assert np.array_equal(X, np.triu(np.array(Pinv, dtype=np.float64)))


def _fraction_inverse(A):
    """Exact inverse by Gauss-Jordan over the rationals."""
    n = len(A)
    W = [list(A[i]) + [Fraction(int(i == j)) for j in range(n)] for i in range(n)]
    for c in range(n):
        p = next(r for r in range(c, n) if W[r][c] != 0)
        W[c], W[p] = W[p], W[c]
        piv = W[c][c]
        W[c] = [v / piv for v in W[c]]
        for r in range(n):
            if r != c and W[r][c] != 0:
                f = W[r][c]
                W[r] = [a - f * b for a, b in zip(W[r], W[c])]
    return [row[n:] for row in W]


def test_exact_rational_4x4(orc):
    """A = R^T R for a rational R with dyadic entries: R is recovered exactly and
    X matches the exact rational inverse."""
    Rq = [[2, 1, -1, Fraction(1, 2)], [0, 4, 2, -3], [0, 0, 1, Fraction(1, 4)], [0, 0, 0, 2]]
    Rq = [[Fraction(v) for v in row] for row in Rq]
    A = [[sum(Rq[k][i] * Rq[k][j] for k in range(4)) for j in range(4)] for i in range(4)]
    Ainv = _fraction_inverse(A)
    R, info = orc.chol(np.array([[float(v) for v in row] for row in A]))
    assert info == 0
    assert np.array_equal(R, np.array([[float(v) for v in row] for row in Rq]))
    X = orc.inv_rows(R)
    np.testing.assert_allclose(full(X), np.array([[float(v) for v in row] for row in Ainv]), rtol=1e-14)


# --------------------------------------------------------------------------
# invariants and independent methods
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [2, 3, 5, 6])
@pytest.mark.parametrize("cplx", [False, True])
def test_gauss_jordan_long_double(orc, n, cplx):
    rng = np.random.default_rng(100 + n + 10 * cplx)
    for _ in range(20):
        A = rand_hpd(rng, n, cplx, shift=0.3)
        R, info = orc.chol(A)
        assert info == 0
        X = full(orc.inv_rows(R))
        Xg = orc.gj(A)
        kappa = np.linalg.cond(A)
        assert np.linalg.norm(X - Xg) / np.linalg.norm(Xg) <= 1e-13 * max(kappa, 1.0)


@pytest.mark.parametrize("n", [3, 9, 24])
@pytest.mark.parametrize("cplx", [False, True])
def test_reconstruction_and_residual(orc, n, cplx):
    rng = np.random.default_rng(7 * n + cplx)
    A = rand_hpd(rng, n, cplx)
    R, info = orc.chol(A)
    assert info == 0
    assert np.all(np.diag(R).real > 0) and np.all(np.diag(R).imag == 0)
    assert np.array_equal(R, np.triu(R))
    u = 2.0 ** -53
    assert np.linalg.norm(np.conj(R).T @ R - A) <= 4 * n * u * np.linalg.norm(A)
    Xu = orc.inv_rows(R)
    assert np.all(np.diag(Xu).imag == 0) and np.all(np.diag(Xu).real > 0)
    X = full(Xu)
    res = np.linalg.norm(A @ X - np.eye(n)) / (np.linalg.norm(A) * np.linalg.norm(X))
    assert res <= 8 * n * u
    # the computed upper half agrees with numpy's LAPACK inverse
    Xn = np.linalg.inv(A)
    assert np.linalg.norm(np.triu(Xn) - Xu) / np.linalg.norm(np.triu(Xn)) <= 50 * n * u * np.linalg.cond(A)


@pytest.mark.parametrize("cplx", [False, True])
def test_orders_and_methods_agree(orc, cplx):
    """Row order and column order give the same bits; Equation Solving (which
    does the forward solve that the proposed method skips) gives the same bits
    as the proposed method, because its b_jj = 1/r_jj and b_ij = 0 (i < j) are
    exactly the s_ij of Eq. 24; Triangular Matrix Operations agrees to rounding."""
    rng = np.random.default_rng(5 + cplx)
    for n in (1, 2, 7, 16, 31):
        A = rand_hpd(rng, n, cplx)
        R, _ = orc.chol(A)
        Xr = orc.inv_rows(R)
        assert np.array_equal(Xr, orc.inv_cols(R))
        assert np.array_equal(Xr, orc.es(R))
        for ex in (False, True):
            Xt = orc.tmo(R, exploit=ex)
            assert np.linalg.norm(Xt - Xr) / np.linalg.norm(Xr) <= 1e-13 * np.linalg.cond(A)


def test_non_pd_info(orc):
    assert orc.chol(np.diag([1.0, -1.0, 1.0]))[1] == 2
    assert orc.chol(np.array([[1.0, 2.0], [2.0, 1.0]]))[1] == 2
    assert orc.chol(np.array([[0.0]]))[1] == 1
    assert orc.chol(np.array([[np.nan, 0.0], [0.0, 1.0]]))[1] == 1
    assert orc.chol(np.array([[1.0, 0.0], [0.0, np.inf]]))[1] == 2
    # a zero pivot after elimination (exactly singular, rank 1)
    assert orc.chol(np.ones((3, 3)))[1] == 2


# --------------------------------------------------------------------------
# operation counts (Table 1)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("cplx", [False, True])
def test_multiply_counts_exact(orc, cplx):
    rng = np.random.default_rng(11)
    for n in range(1, 14):
        A = rand_hpd(rng, n, cplx)
        R, info, c_chol = orc.chol(A, count=True)
        cf = orc.count_closed_form(n)
        assert c_chol == cf["cholesky"] == (n ** 3 - n) // 6
        _, c_inv = orc.inv_rows(R, count=True)
        assert c_inv == cf["proposed_solve"] == sum((n - i) * (n - i + 1) for i in range(1, n + 1))
        assert orc.inv_cols(R, count=True)[1] == c_inv
        assert c_chol + c_inv == cf["proposed"]
        assert c_chol + orc.es(R, count=True)[1] == cf["es"]
        assert c_chol + orc.tmo(R, count=True)[1] == cf["tmo"]
        assert c_chol + orc.tmo(R, exploit=True, count=True)[1] == cf["tmo_exploit"]


def test_table1_leading_terms(orc):
    """The counted multiplies approach Table 1's n^3 coefficients; the reduction
    proposed vs TMO is (2/3 - 1/2) n^3 = 0.1667 n^3, the '16-17%' of Sec. I."""
    g = json.load(open(os.path.join(GOLDEN, "table1.json")))
    lead = {k: Fraction(*v) for k, v in g["leading_coefficient_of_n3"].items()}
    n = 400
    cf = orc.count_closed_form(n)
    rel = 2e-2
    assert abs(cf["es"] / n ** 3 - float(lead["equation_solving"])) < rel * float(lead["equation_solving"])
    assert abs(cf["tmo"] / n ** 3 - float(lead["triangular_matrix_operations"])) < rel
    assert abs(cf["proposed"] / n ** 3 - float(lead["proposed"])) < rel
    assert abs(cf["cholesky"] / n ** 3 - float(lead["cholesky"])) < rel
    saving = (cf["tmo"] - cf["proposed"]) / n ** 3
    lo, hi = g["claimed_reduction_percent"]
    assert lo / 100 <= saving <= hi / 100 + 1e-3
    # the same counts on an actual run, small n, leading coefficient check
    rng = np.random.default_rng(3)
    n = 40
    A = rand_hpd(rng, n, False)
    R, _, c1 = orc.chol(A, count=True)
    c2 = orc.inv_rows(R, count=True)[1]
    assert abs((c1 + c2) / n ** 3 - 0.5) < 0.01


# --------------------------------------------------------------------------
# LDL (Sec. II.A, IV.B)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("cplx", [False, True])
def test_ldl_against_cholesky_and_min_matrix(orc, cplx):
    n = 9
    i = np.arange(1, n + 1)
    A = np.minimum.outer(i, i).astype(np.complex128 if cplx else np.float64)
    R, d, info = orc.ldl(A)
    assert info == 0 and np.array_equal(d, np.ones(n)) and np.array_equal(R, np.triu(np.ones((n, n))))
    rng = np.random.default_rng(9 + cplx)
    A = rand_hpd(rng, 12, cplx)
    R, d, info = orc.ldl(A)
    Rc, _ = orc.chol(A)
    # Cholesky factor = D^(1/2) R_ldl
    np.testing.assert_allclose(np.sqrt(d)[:, None] * R, Rc, rtol=1e-12, atol=1e-13)
    X = orc.ldl_inv(R, d)
    np.testing.assert_allclose(X, orc.inv_rows(Rc), rtol=1e-11, atol=1e-14)
    _, _, _, c = orc.ldl(A, count=True)
    assert c == (12 ** 3 - 12) // 6
    assert orc.ldl_inv(R, d, count=True)[1] == (12 ** 3 - 12) // 3


# --------------------------------------------------------------------------
# adjoint: central differences along Hermitian directions
# --------------------------------------------------------------------------
@pytest.mark.parametrize("cplx", [False, True])
def test_gradient_central_differences(orc, cplx):
    rng = np.random.default_rng(21 + cplx)
    n = 6
    A = rand_hpd(rng, n, cplx)
    W = wl.gaussian((n, n), 5, complex_=cplx)

    def loss(M):
        R, info = orc.chol(M)
        assert info == 0
        return np.real(np.sum(np.conj(W) * full(orc.inv_rows(R)))) if cplx else np.sum(W * full(orc.inv_rows(R)))

    X = full(orc.inv_rows(orc.chol(A)[0]))
    # loss = Re <W, X>; dL/dX = W (complex: W itself in the Re<.,.> pairing)
    dA = orc.grad(X, W)
    h = 1e-6
    for _ in range(4):
        E = rand_hpd(rng, n, cplx, shift=0.0)
        E /= np.linalg.norm(E)
        fd = (loss(A + h * E) - loss(A - h * E)) / (2 * h)
        an = np.real(np.sum(np.conj(dA) * E))
        assert abs(fd - an) <= 1e-7 * max(abs(an), 1e-3)
    # dA is Hermitian
    np.testing.assert_allclose(dA, np.conj(dA).T, atol=1e-14)


# --------------------------------------------------------------------------
# batched driver and layouts
# --------------------------------------------------------------------------
@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("cplx", [False, True])
def test_batch_driver_matches_single(orc, layout, cplx):
    rng = np.random.default_rng(44)
    sizes = rng.integers(1, 12, size=37).astype(np.int32)
    mats = [rand_hpd(rng, int(s), cplx) for s in sizes]
    dense = {}
    for N in np.unique(sizes):
        idx = np.nonzero(sizes == N)[0]
        dense[int(N)] = (idx, np.stack([mats[k] for k in idx]))
    flat, off = wl.pack(dense, sizes, layout, np.complex128 if cplx else np.float64)
    Rf, Xf, info = orc.inv_batch(flat, sizes, off, layout, cplx, want_R=True, nthreads=3)
    assert np.all(info == 0)
    b = wl.Batch(Xf, sizes, off, layout)
    br = wl.Batch(Rf, sizes, off, layout)
    for k, M in enumerate(mats):
        R, _ = orc.chol(M)
        assert np.array_equal(b.matrix(k), orc.inv_rows(R))
        assert np.array_equal(br.matrix(k), R)


# --------------------------------------------------------------------------
# the block form of Sec. IV.A used by the large-order path (a reading)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("n,b", [(37, 8), (64, 16), (50, 50), (9, 4)])
def test_block_form_reading(orc, n, b, cplx):
    """Row block I of R X = S (S's diagonal block is R_II^{-*}, the blocks
    right of it zero) gives, for block rows I = last..first,
        X_I,>I = -R_II^{-1} R_I,>I X_>I,>I
        X_II   =  R_II^{-1} (R_II^{-*} - R_I,>I X_>I,I),  X_>I,I = X_I,>I^*.
    Carried out with numpy's triangular inverses on the oracle's R, it gives
    the oracle's element recurrence to rounding, ragged last block included."""
    rng = np.random.default_rng(900 + n + b + cplx)
    A = rand_hpd(rng, n, cplx)
    R, info = orc.chol(A)
    assert info == 0
    X = np.zeros_like(R)
    starts = list(range(0, n, b))
    for s in reversed(starts):
        e = min(s + b, n)
        Rii_inv = np.linalg.inv(R[s:e, s:e])
        if e < n:
            X[s:e, e:] = -Rii_inv @ (R[s:e, e:] @ X[e:, e:])
            X[e:, s:e] = np.conj(X[s:e, e:]).T
            Z = R[s:e, e:] @ X[e:, s:e]
        else:
            Z = np.zeros((e - s, e - s), dtype=R.dtype)
        X[s:e, s:e] = Rii_inv @ (np.conj(Rii_inv).T - Z)
    ref = full(orc.inv_rows(R))
    kap = np.linalg.cond(A)
    assert np.linalg.norm(X - ref) / np.linalg.norm(ref) <= 50 * n * kap * 2.0 ** -53


@pytest.mark.parametrize("cplx", [False, True])
def test_refinement_indicator_bounds(orc, cplx):
    """The automatic-refinement indicator gamma = max_i a_ii x_ii lies in
    [1, (1 + kappa)^2 / (4 kappa)] with kappa = kappa_2(A): a_ii x_ii =
    (e_i^* A e_i)(e_i^* A^{-1} e_i) is >= 1 by Cauchy-Schwarz and <= the
    Kantorovich bound.  Both ends are reached: gamma = 1 for a diagonal A,
    the upper bound for A = Q diag(1, kappa) Q^T with Q a 45-degree
    rotation."""
    rng = np.random.default_rng(31 + cplx)
    for n in (2, 5, 12, 30):
        for shift in (n, 1e-2, 1e-5):
            A = rand_hpd(rng, n, cplx, shift=shift)
            _, Xu, info = orc.inverse(A)
            assert info == 0
            g = float(np.max(np.real(np.diag(A)) * np.real(np.diag(Xu))))
            kap = np.linalg.cond(A)
            assert 1.0 - 1e-12 <= g <= (1 + kap) ** 2 / (4 * kap) * (1.0 + 1e-9), (g, kap)
    _, Xu, _ = orc.inverse(np.diag([3.0, 7.0, 0.5]))
    assert np.max(np.diag(np.diag([3.0, 7.0, 0.5])) * np.diag(Xu)) == 1.0
    c = np.sqrt(0.5)
    Q = np.array([[c, -c], [c, c]])
    kappa = 1e4
    A = Q @ np.diag([1.0, kappa]) @ Q.T
    _, Xu, _ = orc.inverse(A)
    g = float(np.max(np.diag(A) * np.diag(Xu)))
    assert g == pytest.approx((1 + kappa) ** 2 / (4 * kappa), rel=1e-12)


# --------------------------------------------------------------------------
# the large-matrix forms: threaded Cholesky and inverse, column solves
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 2, 7, 33, 130])
@pytest.mark.parametrize("threads", [1, 3, 8])
def test_threaded_forms_are_the_serial_ones(orc, n, threads):
    """chol_mt / inv_rows_mt split each row's entries over threads: the same
    operations as the pinned serial chol / inv_rows, so the same bits."""
    rng = np.random.default_rng(900 + n)
    A = rand_hpd(rng, n, False)
    R, info = orc.chol(A)
    R2, info2 = orc.chol_mt(A, threads)
    assert info == info2 == 0 and np.array_equal(R, R2)
    assert np.array_equal(orc.inv_rows(R), orc.inv_rows_mt(R, threads))
    # a failing pivot is reported at the same row
    A[n // 2, n // 2] = -1.0
    assert orc.chol_mt(A, threads)[1] == orc.chol(A)[1] == n // 2 + 1


@pytest.mark.parametrize("n", [1, 3, 8, 16, 33])
def test_solve_cols_min_matrix_exact(orc, n):
    """min(i, j) has R = all-ones upper and inverse tridiag(-1, 2, -1) with
    x_nn = 1: every column from the two triangular solves is exact."""
    i = np.arange(1, n + 1)
    A = np.minimum.outer(i, i).astype(np.float64)
    R, info = orc.chol(A)
    T = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    T[-1, -1] = 1.0
    cols = np.arange(n)
    assert np.array_equal(orc.solve_cols(R, cols, 3), T[:, cols].T)


@pytest.mark.parametrize("n", [2, 6, 13, 40])
def test_solve_cols_tridiagonal_closed_form(orc, n):
    """tridiag(-1, 2, -1): (T^-1)_ij = min(i, j)(n + 1 - max(i, j))/(n + 1), 1-based."""
    T = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    R, _ = orc.chol(T)
    i = np.arange(1, n + 1)
    ref = np.minimum.outer(i, i) * (n + 1 - np.maximum.outer(i, i)) / (n + 1)
    cols = np.array([0, n // 2, n - 1])
    got = orc.solve_cols(R, cols)
    assert np.allclose(got, ref[:, cols].T, rtol=0, atol=64 * n * 2.0 ** -52 * np.abs(ref).max())


@pytest.mark.parametrize("n", [2, 4, 6])
def test_solve_cols_gauss_jordan_long_double(orc, n):
    rng = np.random.default_rng(950 + n)
    A = rand_hpd(rng, n, False, shift=0.5)
    R, _ = orc.chol(A)
    ref = orc.gj(A)
    kap = np.linalg.cond(A)
    got = orc.solve_cols(R, np.arange(n), 2)
    assert np.abs(got - ref.T).max() <= 1e-13 * kap * np.abs(ref).max()
