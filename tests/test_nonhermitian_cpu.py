"""Pins for the oracle's non-Hermitian inverse (Sec. III.C: D^{-1} = D^* (D D^*)^{-1})
and the MMSE filter W = (H^* H + s2 I)^{-1} H^* built on the proposed
inverse.  CPU only.

  - D = [[2, 0], [1, 1]]: D D^T = [[4, 2], [2, 2]] has the exact factor
    R = [[2, 1], [0, 1]], so D^{-1} = [[1/2, 0], [-1/2, 1]] comes out exactly;
  - a permutation D: D D^T = I, so D^{-1} = D^T exactly;
  - random real and complex D: D D^{-1} = I and LAPACK's LU inverse agree
    within the bound of a method whose condition number is kappa(D)^2;
  - H with orthonormal columns and s2 = 0: W = H^*; random H, s2 > 0: W
    equals H^* (H H^* + s2 I)^{-1} (the push-through identity, solved by
    LAPACK).
"""
import numpy as np
import pytest

U = 2.0 ** -53


def test_exact_two_by_two(orc):
    D = np.array([[2.0, 0.0], [1.0, 1.0]])
    Di, info = orc.nonhermitian_inverse(D)
    assert info == 0
    assert np.array_equal(Di, np.array([[0.5, 0.0], [-0.5, 1.0]]))


def test_permutation_is_its_transpose(orc):
    P = np.eye(7)[[3, 0, 6, 1, 5, 2, 4]]
    Di, info = orc.nonhermitian_inverse(P)
    assert info == 0
    assert np.array_equal(Di, P.T)


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("n", [3, 8, 15])
def test_random_matches_lu_within_squared_condition(orc, n, cplx):
    rng = np.random.default_rng(40 + n + 100 * cplx)
    D = rng.standard_normal((n, n)) + (1j * rng.standard_normal((n, n)) if cplx else 0)
    Di, info = orc.nonhermitian_inverse(D)
    assert info == 0
    k2 = np.linalg.cond(D) ** 2
    res = np.linalg.norm(D @ Di - np.eye(n)) / np.sqrt(n)
    assert res <= 8 * n * k2 * U, res
    ref = np.linalg.inv(D)
    assert np.linalg.norm(Di - ref) / np.linalg.norm(ref) <= 8 * n * k2 * U


def test_singular_reports_info(orc):
    D = np.array([[1.0, 2.0], [2.0, 4.0]])
    Di, info = orc.nonhermitian_inverse(D)
    assert Di is None and info == 2


@pytest.mark.parametrize("N", [2, 4, 8, 16])
def test_mmse_orthonormal_columns_no_noise(orc, N):
    rng = np.random.default_rng(60 + N)
    G = rng.standard_normal((2 * N, N)) + 1j * rng.standard_normal((2 * N, N))
    Q, _ = np.linalg.qr(G)
    W, info = orc.mmse_filter(Q, 0.0)
    assert info == 0
    assert np.linalg.norm(W - np.conj(Q).T) <= 16 * N * U


@pytest.mark.parametrize("N", [4, 8, 16])
def test_mmse_push_through_identity(orc, N):
    rng = np.random.default_rng(70 + N)
    H = (rng.standard_normal((2 * N, N)) + 1j * rng.standard_normal((2 * N, N))) * np.sqrt(0.5)
    s2 = 0.1
    W, info = orc.mmse_filter(H, s2)
    assert info == 0
    Hh = np.conj(H).T
    # W = H^* (H H^* + s2 I)^{-1}: solve (H H^* + s2 I)^T W^T = (H^*)^T
    M = H @ Hh + s2 * np.eye(2 * N)
    ref = np.linalg.solve(M.T, Hh.T).T
    kap = np.linalg.cond(Hh @ H + s2 * np.eye(N))
    assert np.linalg.norm(W - ref) / np.linalg.norm(ref) <= 64 * N * kap * U
