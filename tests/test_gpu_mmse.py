"""MMSE filters W = (H^* H + s2 I)^{-1} H^* on the GPU (chol_mmse_batched)
against the oracle's mmse_filter, and the non-Hermitian inverse
D^{-1} = D^* (D D^*)^{-1} (Sec. III.C) against the oracle's
nonhermitian_inverse, element by element."""
import numpy as np
import pytest

from paper_1111_4144_gb300 import workloads as wl

from gpu_helpers import TOL64, tol32

pytestmark = pytest.mark.gpu

NP = {"f32": np.float32, "f64": np.float64, "c64": np.complex64, "c128": np.complex128}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1111_4144_gb300 import _lib
    _lib.load()


def _run_flat(tag, H, n, m, hoff, woff, sigma2, **kw):
    import torch
    from paper_1111_4144_gb300 import api
    dev = torch.device("cuda", 0)
    Ht = torch.from_numpy(H.astype(NP[tag])).to(dev)
    W = torch.full_like(Ht, float("nan"))
    W, info = api.mmse(Ht, torch.from_numpy(n).to(dev), torch.from_numpy(m).to(dev), torch.from_numpy(hoff).to(dev),
                       torch.from_numpy(woff).to(dev), int(n.max()), int(m.max()), sigma2=sigma2, W=W, **kw)
    torch.cuda.synchronize()
    return W.cpu().numpy(), info.cpu().numpy()


@pytest.mark.parametrize("sizes", [(3, 4, 8, 16, 23), (1, 3, 4, 8, 16)], ids=["to23", "to16_tiled"])
@pytest.mark.parametrize("tag", ["c64", "c128", "f32", "f64"])
def test_mmse_filter_matches_oracle(orc, tag, sizes):
    """Orders up to 23 (the warp-per-matrix products) and up to 16 with up
    to 32 rows (the register-tiled products), mixed in one flat batch."""
    H, n, m, hoff, woff = wl.mimo_channels(900, sizes=sizes, seed=3100)
    if tag in ("f32", "f64"):
        H = H.real.copy()
    sigma2 = 0.1
    W, info = _run_flat(tag, H, n, m, hoff, woff, sigma2)
    assert np.all(info == 0)
    Hw = H.astype(NP[tag]).astype(np.complex128 if tag.startswith("c") else np.float64)
    for b in range(len(n)):
        N, M = int(n[b]), int(m[b])
        Hb = Hw[hoff[b]:hoff[b] + M * N].reshape(M, N)
        Wo, inf = orc.mmse_filter(Hb, sigma2)
        assert inf == 0
        Wg = W[woff[b]:woff[b] + N * M].reshape(N, M)
        A = np.conj(Hb).T @ Hb + sigma2 * np.eye(N)
        tol = TOL64 if tag in ("f64", "c128") else 2 * float(tol32(np.linalg.cond(A)))
        err = np.linalg.norm(Wg - Wo) / np.linalg.norm(Wo)
        assert err <= tol, (b, N, err, tol)


def test_mmse_with_stated_orders(orc):
    """The channels' order set stated (kernels for those orders only): the
    filters match the oracle; a channel of an order outside the set gets
    info = -1 and leaves the others untouched."""
    H, n, m, hoff, woff = wl.mimo_channels(600, sizes=(4, 8, 16), seed=3101)
    sigma2 = 0.1
    W, info = _run_flat("c64", H, n, m, hoff, woff, sigma2, orders=(4, 8, 16))
    assert np.all(info == 0)
    Hw = H.astype(np.complex64).astype(np.complex128)
    for b in range(0, len(n), 7):
        N, M = int(n[b]), int(m[b])
        Hb = Hw[hoff[b]:hoff[b] + M * N].reshape(M, N)
        Wo, _ = orc.mmse_filter(Hb, sigma2)
        A = np.conj(Hb).T @ Hb + sigma2 * np.eye(N)
        err = np.linalg.norm(W[woff[b]:woff[b] + N * M].reshape(N, M) - Wo) / np.linalg.norm(Wo)
        assert err <= 2 * float(tol32(np.linalg.cond(A))), (b, N, err)
    W2, info2 = _run_flat("c64", H, n, m, hoff, woff, sigma2, orders=(4, 16))
    assert np.all(info2[n == 8] == -1) and np.all(info2[n != 8] == 0)
    from paper_1111_4144_gb300 import _lib as L, api
    assert api.last_device_error() == L.CHOL_ERR_ARG
    keep = np.concatenate([np.arange(woff[b], woff[b] + int(n[b]) * int(m[b])) for b in np.flatnonzero(n != 8)])
    assert np.array_equal(W2[keep], W[keep])


def test_mmse_uniform_tensor_form(orc):
    import torch
    from paper_1111_4144_gb300 import api
    rng = np.random.default_rng(3101)
    batch, M, N = 200, 32, 16
    H = ((rng.standard_normal((batch, M, N)) + 1j * rng.standard_normal((batch, M, N))) * np.sqrt(0.5))
    Ht = torch.from_numpy(H.astype(np.complex64)).cuda()
    W, info = api.mmse(Ht, sigma2=0.5)
    torch.cuda.synchronize()
    W = W.cpu().numpy()
    assert np.all(info.cpu().numpy() == 0) and W.shape == (batch, N, M)
    for b in range(0, batch, 17):
        Hb = H[b].astype(np.complex64).astype(np.complex128)
        Wo, _ = orc.mmse_filter(Hb, 0.5)
        A = np.conj(Hb).T @ Hb + 0.5 * np.eye(N)
        assert np.linalg.norm(W[b] - Wo) / np.linalg.norm(Wo) <= 2 * float(tol32(np.linalg.cond(A)))


@pytest.mark.parametrize("tag", ["c128", "f64", "c64"])
def test_nonhermitian_inverse_through_d_dstar(orc, tag):
    """Sec. III.C: D^{-1} = D^* (D D^*)^{-1}.  With H = D^* (square) and
    s2 = 0 the filter is W = (D D^*)^{-1} D, whose conjugate transpose is
    D^* (D D^*)^{-1} = D^{-1} ((D D^*)^{-1} is Hermitian)."""
    import torch
    from paper_1111_4144_gb300 import api
    rng = np.random.default_rng(3102)
    batch, N = 60, 12
    D = rng.standard_normal((batch, N, N)) + (1j * rng.standard_normal((batch, N, N)) if tag.startswith("c") else 0)
    D = D + 2 * np.sqrt(N) * np.eye(N)  # well conditioned
    D = D.astype(NP[tag])
    Hs = np.conj(np.transpose(D, (0, 2, 1))).copy()
    W, info = api.mmse(torch.from_numpy(Hs).cuda(), sigma2=0.0)
    torch.cuda.synchronize()
    Dinv = np.conj(np.transpose(W.cpu().numpy(), (0, 2, 1)))
    assert np.all(info.cpu().numpy() == 0)
    wide = np.complex128 if tag.startswith("c") else np.float64
    for b in range(batch):
        ref, inf = orc.nonhermitian_inverse(D[b].astype(wide))
        assert inf == 0
        k2 = np.linalg.cond(D[b].astype(wide)) ** 2
        tol = TOL64 if tag in ("f64", "c128") else 2 * float(tol32(k2))
        err = np.linalg.norm(Dinv[b] - ref) / np.linalg.norm(ref)
        assert err <= tol, (b, err, tol)
