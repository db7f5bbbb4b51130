"""chol_inv_batched_host: batches in host memory streamed through the device
in chunks (copies overlapping kernels), checked against the oracle."""
import numpy as np
import pytest

from gpu_helpers import cast_batch, check_errors, oracle_inv, upper_errors
from paper_1111_4144_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _run_host(b, tag, mixed, **kw):
    import torch
    from paper_1111_4144_gb300 import api
    from gpu_helpers import torch_dtype
    A_np, _ = cast_batch(b, tag)
    A_h = torch.from_numpy(A_np).pin_memory()
    X_h = torch.full_like(A_h, float("nan")).pin_memory()
    info_h = torch.full((b.batch,), -7, dtype=torch.int32).pin_memory()
    n_h = torch.from_numpy(b.n).pin_memory() if mixed else None
    off_h = torch.from_numpy(b.off).pin_memory() if mixed else None
    max_n = int(b.n.max())
    h = api.HostInv(torch_dtype(tag), b.batch, max_n, sizes=mixed, layout=b.layout, **kw)
    s = torch.cuda.Stream()
    h(A_h, X_h, n_h, off_h, info_h, stream=s)
    s.synchronize()
    return X_h.numpy(), info_h.numpy()


@pytest.mark.parametrize("tag", ["c64", "f64"])
def test_mixed_packed_many_chunks(orc, tag):
    # 20011 matrices: chunks of 8192 / 8192 / 3627, round-robin over the three slots
    b = (wl.mimo_covariance(20011, sizes=(4, 8, 16), seed=1101, layout=1) if tag == "c64"
         else wl.uneven_loguniform(20011, nmin=2, nmax=20, seed=1101, layout=1))
    X, info = _run_host(b, tag, mixed=True)
    _, Xo, info_o, A_wide = oracle_inv(orc, b, tag)
    assert np.array_equal(info, info_o)
    check_errors(tag, b, A_wide, upper_errors(b, X, Xo), "X")


@pytest.mark.parametrize("tag", ["f32", "c128"])
def test_uniform_dense_full_matrices(orc, tag):
    b = wl.spd_gram_shift(9000, 7, 7.0, seed=1102, layout=0)
    X, info = _run_host(b, tag, mixed=False)
    _, Xo, info_o, A_wide = oracle_inv(orc, b, tag)
    assert np.array_equal(info, info_o)
    check_errors(tag, b, A_wide, upper_errors(b, X, Xo), "X")
    # dense layout: the whole matrix comes back (lower = conjugate mirror)
    for k in (0, 4500, 8999):
        M = X[b.off[k]:b.off[k] + 49].reshape(7, 7)
        assert np.array_equal(np.tril(M, -1), np.conj(np.triu(M, 1)).T)


def test_odd_byte_offsets_and_refinement(orc):
    # FP32 packed order-5 matrices are 60 bytes: chunk starts fall off 16-byte boundaries
    b = wl.uneven_loguniform(17001, nmin=3, nmax=5, seed=1103, layout=1)
    from paper_1111_4144_gb300 import _lib as L
    X, info = _run_host(b, "f32", mixed=True, prec=L.CHOL_PREC_FP32_REFINE, refine_steps=1)
    _, Xo, info_o, A_wide = oracle_inv(orc, b, "f32")
    assert np.array_equal(info, info_o)
    check_errors("f32", b, A_wide, upper_errors(b, X, Xo), "X")


@pytest.mark.parametrize("tag,a_shift,x_shift", [("c64", 3, 5), ("f32", 7, 2)])
def test_host_buffers_off_copy_boundaries(orc, tag, a_shift, x_shift):
    """A_host and X_host as views a few elements into larger pinned buffers
    (off 16- and 128-byte boundaries, A and X at different offsets): the
    results match the oracle, and nothing of X's buffer outside the batch is
    written."""
    import torch
    from paper_1111_4144_gb300 import api
    from gpu_helpers import torch_dtype
    b = (wl.mimo_covariance(20011, sizes=(4, 8, 16), seed=1105, layout=1) if tag == "c64"
         else wl.uneven_loguniform(17001, nmin=3, nmax=5, seed=1105, layout=1))
    A_np, _ = cast_batch(b, tag)
    total = A_np.shape[0]
    A_big = torch.zeros(total + 64, dtype=torch_dtype(tag)).pin_memory()
    X_big = torch.full((total + 64,), 7.0, dtype=torch_dtype(tag)).pin_memory()
    A_big[a_shift:a_shift + total] = torch.from_numpy(A_np)
    A_h, X_h = A_big[a_shift:a_shift + total], X_big[x_shift:x_shift + total]
    info_h = torch.full((b.batch,), -7, dtype=torch.int32).pin_memory()
    h = api.HostInv(torch_dtype(tag), b.batch, int(b.n.max()), sizes=True, layout=b.layout)
    s = torch.cuda.Stream()
    h(A_h, X_h, torch.from_numpy(b.n).pin_memory(), torch.from_numpy(b.off).pin_memory(), info_h, stream=s)
    s.synchronize()
    Xb = X_big.numpy()
    assert np.all(Xb[:x_shift] == 7.0) and np.all(Xb[x_shift + total:] == 7.0)
    _, Xo, info_o, A_wide = oracle_inv(orc, b, tag)
    assert np.array_equal(info_h.numpy(), info_o)
    check_errors(tag, b, A_wide, upper_errors(b, Xb[x_shift:x_shift + total], Xo), "X")


def test_info_of_every_chunk(orc):
    """Non-PD matrices in the first, a middle and the last chunk: info (copied
    back for the whole batch in one piece) flags exactly those, with the
    failing row, and their X is NaN; the others match the oracle."""
    b = wl.mimo_covariance(20011, sizes=(4, 8, 16), seed=1104, layout=1)
    A = b.A.copy()
    bad = [3, 10000, 20010]
    for k in bad:
        A[b.off[k]] = -1.0  # a_11 < 0
    b = wl.Batch(A, b.n, b.off, b.layout)
    X, info = _run_host(b, "c64", mixed=True)
    _, Xo, info_o, A_wide = oracle_inv(orc, b, "c64")
    assert np.array_equal(info, info_o)
    assert sorted(np.flatnonzero(info).tolist()) == bad and np.all(info[bad] == 1)
    for k in bad:
        T = int(b.n[k]) * (int(b.n[k]) + 1) // 2
        assert np.all(np.isnan(np.real(X[b.off[k]:b.off[k] + T])))


def test_rejects_matrices_not_back_to_back():
    import torch
    from paper_1111_4144_gb300 import _lib as L, api
    b = wl.mimo_covariance(100, sizes=(4,), seed=3, layout=1)
    off = b.off.copy() * 2  # gaps between matrices
    A_h = torch.zeros(int(off[-1]) + 10, dtype=torch.complex64).pin_memory()
    X_h = torch.zeros_like(A_h).pin_memory()
    h = api.HostInv(torch.complex64, 100, 4, sizes=True, layout=1)
    with pytest.raises(L.CholError):
        h(A_h, X_h, torch.from_numpy(b.n), torch.from_numpy(off))
