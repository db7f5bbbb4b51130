"""chol_inv_batched_noalloc: the entry point for callers that cannot allocate
device memory (for example code running while a global-mode stream capture
is open, real-time host paths, or plugins whose host application owns all
device memory).  It must give the same results as chol_inv_batched with a
caller workspace, call after call, while using only the library's fixed
scratch array.

This file is named to be collected last, so a run that stops at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_1111_4144_gb300 import workloads as wl

from gpu_helpers import kappas, tol32, upper_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1111_4144_gb300 import _lib
    _lib.load()
    return torch, _lib


def _run(torch, L, b, entry, prec=0, refine_steps=0):
    """Invert batch b (complex64, per-matrix sizes) through one C entry point."""
    dev = torch.device("cuda", 0)
    A = torch.from_numpy(b.A.astype(np.complex64)).to(dev)
    n = torch.from_numpy(b.n).to(dev)
    off = torch.from_numpy(b.off).to(dev)
    X = torch.zeros_like(A)
    info = torch.full((b.batch,), -7, dtype=torch.int32, device=dev)
    max_n = int(b.n.max())
    o = L.opts(prec, refine_steps, 0, b.layout, 0)
    stream = torch.cuda.current_stream().cuda_stream
    if entry == "workspace":
        nbytes = L.chol_workspace_bytes(L.CHOL_CALL_INV, L.CHOL_C64, b.batch, max_n, 1, o)
        ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        st = L.chol_inv_batched(L.CHOL_C64, b.batch, n.data_ptr(), off.data_ptr(), max_n, A.data_ptr(), None,
                                X.data_ptr(), info.data_ptr(), o, ws.data_ptr(), nbytes, stream)
    else:
        st = L.chol_inv_batched_noalloc(L.CHOL_C64, b.batch, n.data_ptr(), off.data_ptr(), max_n, A.data_ptr(),
                                        None, X.data_ptr(), info.data_ptr(), o, stream)
    assert st == L.CHOL_OK, L.status_string(st)
    torch.cuda.synchronize()
    return X.cpu().numpy(), info.cpu().numpy()


def test_noalloc_matches_workspace_entry_two_calls_in_a_row(env):
    torch, L = env
    # two different batches back to back: the second call reuses the scratch
    # array left by the first (different class counts and permutation); the
    # third has 12 orders, whose class kernels run on forked side streams
    b1 = wl.mimo_covariance(6001, sizes=(4, 8, 16), seed=501, layout=1)
    b2 = wl.mimo_covariance(2500, sizes=(3, 11, 16, 2), seed=502, layout=1)
    b3 = wl.mimo_covariance(3000, sizes=tuple(range(1, 13)), seed=503, layout=1)
    for b in (b1, b2, b3):
        Xw, iw = _run(torch, L, b, "workspace")
        Xn, i_n = _run(torch, L, b, "noalloc")
        # the same kernels on the same inputs: the same bits
        assert np.array_equal(iw, i_n) and np.all(i_n == 0)
        assert np.array_equal(Xn, Xw)


def test_noalloc_refinement_matches_workspace_entry(env, orc):
    torch, L = env
    b = wl.mimo_covariance(1200, sizes=(5, 9, 16), seed=504, layout=1)
    Xw, iw = _run(torch, L, b, "workspace", prec=L.CHOL_PREC_FP32_REFINE, refine_steps=1)
    Xn, i_n = _run(torch, L, b, "noalloc", prec=L.CHOL_PREC_FP32_REFINE, refine_steps=1)
    assert np.array_equal(iw, i_n) and np.all(i_n == 0)
    assert np.array_equal(Xn, Xw)
    A_wide = b.A.astype(np.complex64).astype(np.complex128)
    _, Xo, _ = orc.inv_batch(A_wide, b.n, b.off, 1, True)
    err = upper_errors(b, Xn, Xo)
    assert np.all(err <= tol32(kappas(b, A_wide)))


def test_noalloc_rejects_batches_beyond_its_scratch(env):
    torch, L = env
    L.chol_last_device_error(None)  # start from a clear device error word
    o = L.opts(layout=1)
    fake = 0x100000  # never dereferenced: the size check comes first
    st = L.chol_inv_batched_noalloc(L.CHOL_C64, L.CHOL_NOALLOC_MAX_BATCH + 1, fake, fake, 16, fake, None, fake,
                                    None, o, None)
    assert st == L.CHOL_ERR_WORKSPACE
    assert L.chol_last_device_error(None) == L.CHOL_OK
