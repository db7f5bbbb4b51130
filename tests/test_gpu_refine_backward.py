"""GPU tests of the precision options (refinement, FP64 pivots) and of the
adjoint kernel / autograd wrapper, against the CPU oracle."""
import numpy as np
import pytest

from paper_1111_4144_gb300 import workloads as wl

from gpu_helpers import TOL64, U32, cast_batch, kappas, oracle_inv, run_inv, tol32, upper_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1111_4144_gb300 import _lib
    _lib.load()


def _full(Xu):
    return np.triu(Xu) + np.conj(np.triu(Xu, 1)).T


@pytest.mark.parametrize("resid64", [False, True])
@pytest.mark.parametrize("N", [8, 16, 17, 32, 40])
def test_refinement_steps_reduce_error(orc, N, resid64):
    """Refinement with the residual in compensated FP32 pairs (default) or
    in FP64 (CHOL_FLAG_RESIDUAL_FP64): each step cuts the error tenfold or
    reaches FP32 accuracy."""
    from paper_1111_4144_gb300 import _lib as L
    b = wl.fixed_kappa(60, N, 1e4, seed=70 + N, layout=0)
    _, Xo, _, A_wide = oracle_inv(orc, b, "f32")
    errs = []
    flags = L.CHOL_FLAG_RESIDUAL_FP64 if resid64 else 0
    for steps in (0, 1, 2):
        X, info, _ = run_inv(b, "f32", mixed=False, prec=L.CHOL_PREC_FP32_REFINE, refine_steps=steps, flags=flags)
        assert np.all(info == 0)
        errs.append(upper_errors(b, X, Xo))
    k = kappas(b, A_wide)
    assert np.all(errs[0] <= tol32(k))
    assert np.all(errs[1] <= np.maximum(errs[0] / 10, 64 * U32))
    assert np.all(errs[2] <= 64 * U32), f"max {errs[2].max()}"


def test_refinement_automatic_selects_ill_conditioned(orc):
    from paper_1111_4144_gb300 import _lib as L
    N = 12
    easy = wl.fixed_kappa(40, N, 10.0, seed=5, layout=1)
    hard = wl.fixed_kappa(40, N, 1e6, seed=6, layout=1)
    # interleave the two sets into one packed batch
    A = np.concatenate([easy.A, hard.A])
    n = np.concatenate([easy.n, hard.n])
    off, _ = wl.layout_offsets(n, 1)
    b = wl.Batch(A, n, off, 1)
    X0, _, _ = run_inv(b, "f32", mixed=False)
    Xa, info, _ = run_inv(b, "f32", mixed=False, prec=L.CHOL_PREC_FP32_REFINE, refine_steps=-1)
    assert np.all(info == 0)
    _, Xo, _, A_wide = oracle_inv(orc, b, "f32")
    bb = wl.Batch(A_wide, n, off, 1)
    bx = wl.Batch(X0.astype(np.float64), n, off, 1)
    for k in range(b.batch):
        gamma = np.max(np.diag(bb.matrix(k)) * np.diag(bx.matrix(k)))
        T = N * (N + 1) // 2
        changed = not np.array_equal(X0[off[k]:off[k] + T], Xa[off[k]:off[k] + T])
        assert changed == (gamma > 4096.0), (k, gamma)
    err0 = upper_errors(b, X0, Xo)
    erra = upper_errors(b, Xa, Xo)
    hard_idx = np.arange(40, 80)
    assert np.all(erra[hard_idx] < err0[hard_idx] / 10)


@pytest.mark.parametrize("tag", ["f32", "c64"])
@pytest.mark.parametrize("N", [6, 16, 24, 48])
def test_pivot64_flag(orc, tag, N):
    from paper_1111_4144_gb300 import _lib as L
    if tag == "c64":
        b = wl.mimo_covariance(100, sizes=(N,), seed=9, layout=1, shuffle=False)
    else:
        b = wl.fixed_kappa(100, N, 1e3, seed=9, layout=1)
    X, info, R = run_inv(b, tag, mixed=False, want_R=True, flags=L.CHOL_FLAG_PIVOT64)
    Ro, Xo, info_o, A_wide = oracle_inv(orc, b, tag)
    assert np.array_equal(info, info_o)
    tol = tol32(kappas(b, A_wide))
    assert np.all(upper_errors(b, X, Xo) <= tol)
    assert np.all(upper_errors(b, R, Ro) <= tol)


@pytest.mark.parametrize("tag", ["f32", "f64", "c64", "c128"])
@pytest.mark.parametrize("N", [1, 5, 16, 32, 45])
@pytest.mark.parametrize("xlayout", [0, 1])
def test_backward_matches_oracle(orc, tag, N, xlayout):
    import torch
    from paper_1111_4144_gb300 import api
    cplx = tag.startswith("c")
    batch = 24
    b = wl.fixed_kappa(batch, N, 1e2, seed=40 + N, layout=xlayout) if not cplx else \
        wl.mimo_covariance(batch, sizes=(N,), seed=40 + N, layout=xlayout, shuffle=False)
    A_np, A_wide = cast_batch(b, tag)
    _, Xo, _ = orc.inv_batch(A_wide, b.n, b.off, xlayout, cplx)
    # the forward X in the working precision, as the GPU would have produced it
    Xw = Xo.astype(A_np.dtype)
    G = wl.gaussian((batch, N, N), 77, complex_=cplx).astype(A_np.dtype)
    dev = torch.device("cuda", 0)
    Xt = torch.from_numpy(Xw).to(dev)
    Gt = torch.from_numpy(G).to(dev)
    if xlayout == 0:
        dA = api.backward(Xt.view(batch, N, N), Gt)
    else:
        dA = api.backward(Xt, Gt, max_n=N, layout=1)
    torch.cuda.synchronize()
    dA = dA.cpu().numpy().reshape(batch, N, N)
    bx = wl.Batch(Xw.astype(np.complex128 if cplx else np.float64), b.n, b.off, xlayout)
    for k in range(batch):
        Xf = _full(bx.matrix(k))
        ref = orc.grad(Xf, G[k].astype(Xf.dtype))
        err = np.linalg.norm(dA[k] - ref) / np.linalg.norm(ref)
        if tag in ("f64", "c128"):
            assert err <= TOL64, err
        else:
            kap = np.linalg.cond(Xf)
            assert err <= 2 * tol32(kap) + 32 * U32, err
        np.testing.assert_allclose(dA[k], np.conj(dA[k]).T, rtol=0, atol=1e-12 * np.abs(dA[k]).max())


@pytest.mark.parametrize("dtype", ["float64", "complex128"])
def test_autograd_gradcheck(dtype):
    import torch
    from paper_1111_4144_gb300 import api
    torch.manual_seed(0)
    dev = torch.device("cuda", 0)
    N, batch = 4, 3
    dt = getattr(torch, dtype)
    B = torch.randn(batch, N, N, dtype=dt)
    A = (B @ B.mH + N * torch.eye(N, dtype=dt)).to(dev).requires_grad_(True)
    f = lambda M: api.inv_autograd(M)[0]
    assert torch.autograd.gradcheck(f, (A,), eps=1e-6, atol=1e-7, rtol=1e-5)


def test_autograd_fp32_against_fp64_central_differences(orc):
    """The differentiation workload: N = 32, kappa = 1e2, loss = sum(W o X).
    The FP32 GPU gradient (Hermitian form) against FP64 central differences
    of the oracle along random symmetric directions."""
    import torch
    from paper_1111_4144_gb300 import api
    N, batch = 32, 8
    b = wl.fixed_kappa(batch, N, 1e2, seed=1003, layout=0)
    A32 = b.A.astype(np.float32).reshape(batch, N, N)
    W = wl.gaussian((batch, N, N), 1003)
    dev = torch.device("cuda", 0)
    A = torch.from_numpy(A32).to(dev).requires_grad_(True)
    X, _ = api.inv_autograd(A)
    loss = (torch.from_numpy(W.astype(np.float32)).to(dev) * X).sum()
    loss.backward()
    g_upper = A.grad.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(3)
    h = 1e-6
    for k in range(batch):
        Ak = A32[k].astype(np.float64)
        Ak = np.triu(Ak) + np.triu(Ak, 1).T

        def loss_k(M):
            R, info = orc.chol(M)
            assert info == 0
            return float(np.sum(W[k] * _full(orc.inv_rows(R))))

        for _ in range(2):
            E = rng.standard_normal((N, N))
            E = (E + E.T) / 2
            E /= np.linalg.norm(E)
            fd = (loss_k(Ak + h * E) - loss_k(Ak - h * E)) / (2 * h)
            # the upper-parameter gradient pairs with the upper triangle of E
            an = float(np.sum(np.triu(g_upper[k]) * np.triu(E)))
            assert abs(fd - an) <= (2 * tol32(1e2) + 32 * U32) * max(abs(fd), 1.0), (fd, an)


@pytest.mark.parametrize("N", [6, 16, 24, 33])
def test_refinement_complex_both_residuals(orc, N):
    """Complex64 refinement, both residual forms, against the oracle."""
    from paper_1111_4144_gb300 import _lib as L
    b = wl.mimo_covariance(48, sizes=(N,), sigma2=1e-3, seed=80 + N, layout=1, shuffle=False)
    _, Xo, _, A_wide = oracle_inv(orc, b, "c64")
    X0, _, _ = run_inv(b, "c64", mixed=False)
    e0 = upper_errors(b, X0, Xo)
    for flags in (0, L.CHOL_FLAG_RESIDUAL_FP64):
        X, info, _ = run_inv(b, "c64", mixed=False, prec=L.CHOL_PREC_FP32_REFINE, refine_steps=2, flags=flags)
        assert np.all(info == 0)
        e = upper_errors(b, X, Xo)
        assert np.all(e <= np.maximum(e0 / 10, 64 * U32)), (flags, e.max(), e0.max())


@pytest.mark.parametrize("tag,nmax", [("f32", 16), ("f32", 32), ("c64", 16), ("c64", 32)])
def test_refinement_mixed_orders(orc, tag, nmax):
    """Refinement of a batch of mixed orders 1..nmax (the order-16 and
    order-32 tiles, zero padding of every smaller order, packed layout): two
    steps reach FP32 accuracy or cut the error tenfold, matrix by matrix."""
    from paper_1111_4144_gb300 import _lib as L
    b = wl.uneven_loguniform(300, nmin=1, nmax=nmax, decades=3.0, seed=90 + nmax, layout=1)
    if tag == "c64":
        b = wl.Batch(b.A.astype(np.complex128), b.n, b.off, b.layout)
    _, Xo, _, A_wide = oracle_inv(orc, b, tag)
    X0, _, _ = run_inv(b, tag, mixed=True)
    X, info, _ = run_inv(b, tag, mixed=True, prec=L.CHOL_PREC_FP32_REFINE, refine_steps=2)
    assert np.all(info == 0)
    e0 = upper_errors(b, X0, Xo)
    e = upper_errors(b, X, Xo)
    assert np.all(e <= np.maximum(e0 / 10, 64 * U32)), (e.max(), e0.max())
