"""The LDL form (CHOL_FLAG_LDL; Sec. II.A Eqs. 9-11, Sec. IV.B Eqs. 25-29)
against the oracle: X = A^{-1} as for Cholesky, and the unit upper factor R
with d_i on its diagonal against the oracle's LDL decomposition."""
import numpy as np
import pytest

from gpu_helpers import cast_batch, check_errors, kappas, oracle_inv, run_inv, tol32, upper_errors, TOL64
from paper_1111_4144_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
TAGS = ["f32", "f64", "c64", "c128"]


def _batch(tag, kind):
    if kind == "mimo":
        b = wl.mimo_covariance(2000, sizes=(4, 8, 16), seed=2101, layout=1)
    elif kind == "orders_1_32_packed":
        # every order of the thread-per-matrix and group kernels, several
        # chunks of the order-1 lane kernel's CTA
        b = wl.uneven_loguniform(1500, nmin=1, nmax=32, seed=2103, layout=1)
        assert set(b.n.tolist()) == set(range(1, 33))
    else:
        b = wl.uneven_loguniform(300, nmin=1, nmax=64, seed=2102, layout=0)
    if tag in ("f32", "f64") and np.iscomplexobj(b.A):
        b = wl.Batch(b.A.real.copy(), b.n, b.off, b.layout)
    return b


@pytest.mark.parametrize("kind", ["mimo", "uneven", "orders_1_32_packed"])
@pytest.mark.parametrize("tag", TAGS)
def test_ldl_inverse_parity(orc, tag, kind):
    from paper_1111_4144_gb300 import _lib as L
    b = _batch(tag, kind)
    X, info, R = run_inv(b, tag, mixed=True, want_R=True, flags=L.CHOL_FLAG_LDL)
    _, Xo, info_o, A_wide = oracle_inv(orc, b, tag)
    assert np.array_equal(info, info_o)
    check_errors(tag, b, A_wide, upper_errors(b, X, Xo), "X (LDL)")
    # R: unit upper off the diagonal, d_i on it (Eqs. 10-11)
    bb = wl.Batch(A_wide, b.n, b.off, b.layout)
    Rb = wl.Batch(np.asarray(R).astype(A_wide.dtype), b.n, b.off, b.layout)
    # the factor at the same tolerances as X: relative Frobenius error of d and
    # of R's strictly upper part, FP64 <= 1e-11, FP32 <= max(1e-7 kappa, 2.4e-7)
    kap = kappas(b, A_wide)
    for k in range(0, b.batch, max(1, b.batch // 60)):
        A = bb.matrix(k)
        A = np.triu(A) + np.conj(np.triu(A, 1)).T
        Ro, d, inf = orc.ldl(A)
        assert inf == 0
        tol = TOL64 if tag in ("f64", "c128") else float(tol32(kap[k]))
        Rg = Rb.matrix(k)
        dg = np.real(np.diag(Rg))
        assert np.linalg.norm(dg - d) / np.linalg.norm(d) <= tol, (k, np.linalg.norm(dg - d) / np.linalg.norm(d))
        off_g, off_o = np.triu(Rg, 1), np.triu(Ro, 1)
        if A.shape[0] > 1:
            err = np.linalg.norm(off_g - off_o) / np.linalg.norm(off_o)
            assert err <= tol, (k, err, tol)


@pytest.mark.parametrize("tag", ["f64", "c64"])
def test_ldl_non_pd_info(orc, tag):
    from paper_1111_4144_gb300 import _lib as L
    b = _batch(tag, "mimo")
    A = b.A.copy()
    k = 5
    o, n = int(b.off[k]), int(b.n[k])
    A[o] = -1.0  # a_11 < 0: d_1 fails
    b = wl.Batch(A, b.n, b.off, b.layout)
    X, info, _ = run_inv(b, tag, mixed=True, flags=L.CHOL_FLAG_LDL)
    assert info[k] == 1 and np.count_nonzero(info) == 1
    seg = X[o:o + n * (n + 1) // 2]
    assert np.all(np.isnan(np.real(seg)))


def test_ldl_rejects_fp64_pivots():
    import torch
    from paper_1111_4144_gb300 import _lib as L, api
    A = torch.eye(4, dtype=torch.float32, device="cuda").reshape(1, 4, 4).contiguous()
    with pytest.raises(L.CholError):
        api.inv(A, flags=L.CHOL_FLAG_LDL | L.CHOL_FLAG_PIVOT64)
