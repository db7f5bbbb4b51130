"""The PyTorch binding rejects mismatched output buffers and short per-matrix
arrays before it calls the library (these checks run on the host; the C call
is replaced by a stub that records that it was reached, and CPU tensors stand
in for device ones)."""
import types

import pytest
import torch

from paper_1111_4144_gb300 import _lib, api


@pytest.fixture()
def stubbed(monkeypatch):
    _lib.load(build_if_missing=True)
    calls = []

    def stub(name):
        def f(*args):
            calls.append(name)
            return 0
        return f

    for name in ("chol_inv_batched", "chol_factor_batched", "chol_inv_backward"):
        monkeypatch.setattr(_lib, name, stub(name))
    monkeypatch.setattr(api, "_need_cuda", lambda *ts: None)
    return calls


STREAM = types.SimpleNamespace(cuda_stream=0)


def test_inv_accepts_matching_buffers(stubbed):
    A = torch.zeros(5, 4, 4)
    api.inv(A, X=torch.zeros_like(A), R=torch.zeros_like(A), want_R=True,
            info=torch.zeros(5, dtype=torch.int32), stream=STREAM)
    assert stubbed == ["chol_inv_batched"]


@pytest.mark.parametrize("bad", ["X_short", "X_dtype", "R_short", "info_short", "info_dtype", "off_short"])
def test_inv_rejects_mismatched_buffers(stubbed, bad):
    A = torch.zeros(5, 4, 4)
    kw = {"stream": STREAM}
    n = off = None
    if bad == "X_short":
        kw["X"] = torch.zeros(4, 4, 4)
    elif bad == "X_dtype":
        kw["X"] = torch.zeros(5, 4, 4, dtype=torch.float64)
    elif bad == "R_short":
        kw["R"] = torch.zeros(5 * 16 - 1)
        kw["want_R"] = True
    elif bad == "info_short":
        kw["info"] = torch.zeros(4, dtype=torch.int32)
    elif bad == "info_dtype":
        kw["info"] = torch.zeros(5, dtype=torch.int64)
    else:
        A = torch.zeros(80)
        n = torch.full((5,), 4, dtype=torch.int32)
        off = torch.arange(4, dtype=torch.int64) * 16
    with pytest.raises(ValueError):
        api.inv(A, n, off, 4, **kw)
    assert stubbed == []


def test_factor_and_backward_checks(stubbed):
    A = torch.zeros(3, 5, 5)
    with pytest.raises(ValueError):
        api.factor(A, R=torch.zeros(3, 5, 4), stream=STREAM)
    with pytest.raises(ValueError):
        api.backward(A, torch.zeros_like(A), dA=torch.zeros(3, 5, 5, dtype=torch.float64), stream=STREAM)
    with pytest.raises(ValueError):
        api.backward(torch.zeros(2, 5, 5), torch.zeros_like(A), stream=STREAM)
    assert stubbed == []
    api.factor(A, R=torch.zeros_like(A), stream=STREAM)
    api.backward(A, torch.zeros_like(A), dA=torch.zeros_like(A), stream=STREAM)
    assert stubbed == ["chol_factor_batched", "chol_inv_backward"]


@pytest.mark.parametrize("bad", [None, "A_dtype", "X_short", "info_short", "n_dtype", "off_short"])
def test_host_inv_checks(monkeypatch, bad):
    _lib.load(build_if_missing=True)
    calls = []
    monkeypatch.setattr(_lib, "chol_inv_batched_host", lambda *a: calls.append(1) or 0)
    h = api.HostInv(torch.complex64, 10, 4, sizes=True, layout=api.LAYOUT_PACKED, device=torch.device("cpu"))
    A = torch.zeros(100, dtype=torch.complex64)
    X = torch.zeros_like(A)
    n = torch.full((10,), 4, dtype=torch.int32)
    off = torch.arange(10, dtype=torch.int64) * 10
    info = torch.zeros(10, dtype=torch.int32)
    if bad == "A_dtype":
        A, X = A.to(torch.complex128), X.to(torch.complex128)
    elif bad == "X_short":
        X = torch.zeros(99, dtype=torch.complex64)
    elif bad == "info_short":
        info = torch.zeros(9, dtype=torch.int32)
    elif bad == "n_dtype":
        n = n.to(torch.int64)
    elif bad == "off_short":
        off = off[:9]
    if bad is None:
        h(A, X, n, off, info, stream=STREAM)
        assert calls == [1]
    else:
        with pytest.raises(ValueError):
            h(A, X, n, off, info, stream=STREAM)
        assert calls == []
