"""The seeded input generators hold their stated recipes: order shares and
shuffling, storage back to back, and the spectra (Hermitian positive definite
with the stated eigenvalues or bounds) that the workloads are defined by."""
import numpy as np
import pytest

from paper_1111_4144_gb300 import workloads as wl


def _dense(b, k):
    """Matrix k of a batch as a full Hermitian square."""
    N = int(b.n[k])
    if b.layout == wl.LAYOUT_DENSE:
        return b.A[b.off[k]:b.off[k] + N * N].reshape(N, N)
    M = np.zeros((N, N), dtype=b.A.dtype)
    iu = np.triu_indices(N)
    M[iu] = b.A[b.off[k]:b.off[k] + wl.tri(N)]
    return M + np.conj(np.triu(M, 1)).T


def _back_to_back(b):
    per = b.n.astype(np.int64) ** 2 if b.layout == wl.LAYOUT_DENSE else wl.tri(b.n.astype(np.int64))
    return b.off[0] == 0 and np.array_equal(b.off[1:], np.cumsum(per)[:-1]) and b.A.size == per.sum()


def test_mimo_covariance_recipe():
    b = wl.mimo_covariance(3001, sizes=(4, 8, 16), sigma2=0.1, seed=21)
    # equal shares, the first size taking the remainder, in a shuffled order
    assert [int((b.n == s).sum()) for s in (4, 8, 16)] == [1001, 1000, 1000]
    assert not np.all(np.diff(b.n) >= 0)
    assert _back_to_back(b)
    # A = H^* H + 0.1 I with H 2N x N of iid CN(0,1): eigenvalues >= 0.1, E[a_ii] = 2N + 0.1
    for s in (4, 8, 16):
        idx = np.flatnonzero(b.n == s)
        ev = np.linalg.eigvalsh(np.stack([_dense(b, k) for k in idx[:200]]))
        assert ev.min() >= 0.1 * (1 - 1e-9)
        diag = np.concatenate([np.real(np.diagonal(_dense(b, k))) for k in idx])
        assert diag.mean() == pytest.approx(2 * s + 0.1, rel=0.03)
    # the same seed gives the same batch
    again = wl.mimo_covariance(3001, sizes=(4, 8, 16), sigma2=0.1, seed=21)
    assert np.array_equal(again.A, b.A) and np.array_equal(again.n, b.n)


def test_uneven_loguniform_recipe():
    b = wl.uneven_loguniform(400, nmin=2, nmax=64, decades=3.0, seed=22)
    assert b.n.min() >= 2 and b.n.max() <= 64 and len(np.unique(b.n)) > 40
    assert _back_to_back(b)
    for k in range(0, 400, 7):
        A = _dense(b, k)
        assert np.array_equal(A, A.T)
        ev = np.linalg.eigvalsh(A)
        assert ev.min() >= 1 - 1e-9 and ev.max() <= 1e3 * (1 + 1e-9)
        assert b.kappa[k] == pytest.approx(ev.max() / ev.min(), rel=1e-8)


def test_fixed_kappa_is_exact():
    b = wl.fixed_kappa(20, 32, 1e2, seed=23)
    for k in range(20):
        ev = np.linalg.eigvalsh(_dense(b, k))
        assert ev.min() == pytest.approx(1.0, rel=1e-10) and ev.max() == pytest.approx(100.0, rel=1e-10)


def test_log_spaced_spectrum():
    N = 50
    b = wl.log_spaced(N, decades=4.0, seed=24)
    ev = np.linalg.eigvalsh(_dense(b, 0))
    assert ev == pytest.approx(10.0 ** (4.0 * np.arange(N) / (N - 1)), rel=1e-9)


def test_gram_shift_recipe():
    b = wl.spd_gram_shift(2000, 8, 8.0, seed=25)
    assert _back_to_back(b)
    A = np.stack([_dense(b, k) for k in range(2000)])
    assert np.linalg.eigvalsh(A).min() >= 8.0 * (1 - 1e-12)
    # B B^T + 8 I with B iid N(0,1): E[a_ii] = N + 8
    assert np.diagonal(A, axis1=1, axis2=2).mean() == pytest.approx(16.0, rel=0.03)


def test_mimo_channels_layout_and_moments():
    H, n, m, hoff, woff = wl.mimo_channels(3000, sizes=(4, 8, 16), seed=26)
    assert np.array_equal(m, 2 * n)
    per = m.astype(np.int64) * n
    assert hoff[0] == 0 and np.array_equal(hoff[1:], np.cumsum(per)[:-1]) and H.size == per.sum()
    assert np.array_equal(hoff, woff)
    # iid CN(0,1): E h = 0, E |h|^2 = 1, real and imaginary parts of variance 1/2
    assert abs(H.mean()) < 0.01 and np.mean(np.abs(H) ** 2) == pytest.approx(1.0, rel=0.01)
    assert np.var(H.real) == pytest.approx(0.5, rel=0.02)


@pytest.mark.parametrize("complex_", [False, True])
def test_bordered_cancellation_last_pivot(complex_):
    """The last pivot's argument (Eq. 3) is `ratio` FP32 ulps of a_NN: a
    cancellation that FP32 pivots cannot resolve, FP64 ones can."""
    ratio = 16.0
    b = wl.bordered_cancellation(30, 12, ratio=ratio, seed=27, complex_=complex_)
    for k in range(30):
        A = _dense(b, k)
        R = np.linalg.cholesky(A).conj().T  # upper factor, A = R^* R
        t = abs(R[-1, -1]) ** 2             # a_NN minus the sum of |r_kN|^2 over k < N
        assert t / np.real(A[-1, -1]) == pytest.approx(ratio * 2.0 ** -24 / (1 + ratio * 2.0 ** -24), rel=1e-6)
        assert t / np.real(A[-1, -1]) < 2.0 ** -10
        # every entry but a_NN is exact in FP32
        off_diag = A.copy()
        off_diag[-1, -1] = 0
        assert np.array_equal(off_diag.astype(np.complex64 if complex_ else np.float32), off_diag)
