"""GPU parity at the full sizes of the four batched workloads, each launched
as the benchmark launches it.

  - 4,096 real FP64 matrices of order 8, A = B B^T + 8 I: small enough for
    the oracle to check every matrix (R and X).
  - 1,048,576 complex64 MIMO covariances of orders 4, 8 and 16, packed, one
    CUDA-graph replay after autotuning.
  - 262,144 real FP32 matrices with orders uniform on 2..64, lambda
    log-uniform on [1, 1e3], dense, one call with per-matrix orders.
  - 65,536 real FP32 matrices of order 32 with kappa = 1e2, forward and
    adjoint through torch.autograd with loss = sum(W o X).

The oracle checks a seeded sample of matrices one by one (first and last
included); every matrix is checked against properties that hold at any
size: info = 0, every output element written and finite, and
x_ii a_ii >= 1 for an HPD matrix (Cauchy-Schwarz on e_i), here with slack
for rounding.
"""
import numpy as np
import pytest

from paper_1111_4144_gb300 import workloads as wl

from gpu_helpers import (TOL64, U32, cast_batch, check_errors, diagonal_positions, kappas, oracle_inv, run_inv,
                         sub_batch, tol32, upper_errors)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1111_4144_gb300 import _lib
    _lib.load()


def sample_indices(batch, count, seed):
    idx = np.random.default_rng(seed).choice(batch, size=min(count, batch), replace=False)
    return np.unique(np.concatenate([idx, [0, batch - 1]]))


def check_sample(orc, b, tag, idx, X_flat):
    """Oracle parity on matrices idx of the batch (inputs rounded to the
    working precision on both sides)."""
    sb = sub_batch(b, idx)
    sx = sub_batch(b, idx, X_flat)
    _, Xo, info_o, A_wide = oracle_inv(orc, sb, tag)
    assert np.all(info_o == 0)
    check_errors(tag, sb, A_wide, upper_errors(sb, sx.A, Xo), f"X (sample of {len(idx)})")


def check_diagonal(b, A_np, X_np):
    pos = diagonal_positions(b)
    xa = np.real(X_np[pos]).astype(np.float64) * np.real(A_np[pos]).astype(np.float64)
    assert np.all(np.isfinite(xa))
    assert xa.min() >= 0.5, f"x_ii a_ii = {xa.min():.3g}"


def test_gram_shift_fp64_order8_every_matrix(orc):
    b = wl.spd_gram_shift(4096, 8, 8.0, seed=1000, layout=wl.LAYOUT_DENSE)
    X, info, R = run_inv(b, "f64", mixed=False, want_R=True)
    Ro, Xo, info_o, A_wide = oracle_inv(orc, b, "f64")
    assert np.all(info == 0) and np.all(info_o == 0)
    for what, got, ref in (("X", X, Xo), ("R", R, Ro)):
        err = upper_errors(b, got, ref)
        assert err.max() <= TOL64, f"{what}: worst relative error {err.max():.3g}"
    # R's strictly lower part is written as zero in the dense layout
    Rd = R.reshape(4096, 8, 8)
    assert np.all(np.tril(Rd, -1) == 0)


def test_mimo_c64_x1048576_graph_replay(orc, tmp_path):
    import torch
    from paper_1111_4144_gb300 import api
    b = wl.mimo_covariance(1 << 20, sizes=(4, 8, 16), sigma2=0.1, seed=1001, layout=wl.LAYOUT_PACKED)
    A_np, _ = cast_batch(b, "c64")
    dev = torch.device("cuda", 0)
    api.autotune(torch.complex64, 16, layout=api.LAYOUT_PACKED, batch=65536,
                 cache_path=str(tmp_path / "tune.txt"))
    A = torch.from_numpy(A_np).to(dev)
    X = torch.full_like(A, complex(float("nan"), float("nan")))
    n = torch.from_numpy(b.n).to(dev)
    off = torch.from_numpy(b.off).to(dev)
    plan = api.Plan(A, X, n, off, 16, layout=api.LAYOUT_PACKED, fixed_orders=True)
    plan.launch()
    torch.cuda.synchronize()
    X1 = X.cpu().numpy()
    info = plan.info.cpu().numpy()
    plan.launch()
    torch.cuda.synchronize()
    X2 = X.cpu().numpy()
    plan.close()
    assert np.all(info == 0)
    assert np.all(np.isfinite(X1)), "an element of X was not written"
    assert np.array_equal(X1, X2), "a second replay changed X"
    check_diagonal(b, A_np, X1)
    check_sample(orc, b, "c64", sample_indices(b.batch, 3000, 11), X1)


def test_uneven_f32_x262144_orders_2_to_64(orc):
    import torch
    from paper_1111_4144_gb300 import api
    b = wl.uneven_loguniform(1 << 18, nmin=2, nmax=64, seed=1002, layout=wl.LAYOUT_DENSE)
    A_np, _ = cast_batch(b, "f32")
    dev = torch.device("cuda", 0)
    A = torch.from_numpy(A_np).to(dev)
    X = torch.full_like(A, float("nan"))
    n = torch.from_numpy(b.n).to(dev)
    off = torch.from_numpy(b.off).to(dev)
    _, info = api.inv(A, n, off, 64, layout=api.LAYOUT_DENSE, fill_lower=True, X=X)
    torch.cuda.synchronize()
    del A
    X_np = X.cpu().numpy()
    assert np.all(info.cpu().numpy() == 0)
    # fill_lower: every element of every matrix is written
    assert np.all(np.isfinite(X_np)), "an element of X was not written"
    check_diagonal(b, A_np, X_np)
    check_sample(orc, b, "f32", sample_indices(b.batch, 1024, 12), X_np)


def test_autograd_f32_x65536_order32(orc):
    import torch
    from paper_1111_4144_gb300 import api
    batch, N = 1 << 16, 32
    b = wl.fixed_kappa(batch, N, 1e2, seed=1003, layout=wl.LAYOUT_DENSE)
    A_np, _ = cast_batch(b, "f32")
    W = wl.gaussian((batch, N, N), 1003).astype(np.float32)
    dev = torch.device("cuda", 0)
    A = torch.from_numpy(A_np.reshape(batch, N, N)).to(dev).requires_grad_(True)
    X, info = api.inv_autograd(A)
    loss = (torch.from_numpy(W).to(dev) * X).sum()
    loss.backward()
    torch.cuda.synchronize()
    assert np.all(info.cpu().numpy() == 0)
    X_np = X.detach().cpu().numpy().reshape(-1)
    g = A.grad.cpu().numpy()
    assert np.all(np.isfinite(X_np)) and np.all(np.isfinite(g))
    check_diagonal(b, A_np, X_np)
    idx = sample_indices(batch, 256, 13)
    check_sample(orc, b, "f32", idx, X_np)
    # the gradient with respect to the upper triangle (2 dA_ij above the
    # diagonal, dA_ii on it) against the oracle's adjoint of its own X
    sb = sub_batch(b, idx)
    _, A_wide = cast_batch(sb, "f32")
    _, Xo, _ = orc.inv_batch(A_wide, sb.n, sb.off, sb.layout, False, fill_lower=True)
    Xo = Xo.reshape(len(idx), N, N)
    kap = kappas(sb, A_wide)
    for k, j in enumerate(idx):
        dA = orc.grad(Xo[k], W[j].astype(np.float64))
        ref = np.triu(2.0 * dA, 1) + np.diag(np.diag(dA))
        err = np.linalg.norm(np.triu(g[j]) - ref) / np.linalg.norm(ref)
        assert err <= 2 * tol32(kap[k]) + 32 * U32, (j, err)
        assert np.all(np.tril(g[j], -1) == 0)
