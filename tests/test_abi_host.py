"""The C-ABI library on the host: it builds, loads, exports every symbol that
include/cholinv.h declares, and rejects invalid arguments before launching
anything (these calls touch no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cholinv.h")


@pytest.fixture(scope="module")
def L():
    from paper_1111_4144_gb300 import _lib
    _lib.load(build_if_missing=True)
    return _lib


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(chol_[a-z0-9_]+)\s*\(", src)))


def test_header_symbols_exported(L):
    names = declared_functions()
    assert len(names) >= 10
    lib = ctypes.CDLL(L.lib_path())
    for name in names:
        assert hasattr(lib, name), f"{name} declared in cholinv.h but not exported"
    # the binding covers every declared entry point under the same name
    assert set(names) <= set(L.SIGNATURES)


def test_status_strings_and_version(L):
    assert L.status_string(L.CHOL_OK) == "success"
    for st in (L.CHOL_ERR_ARG, L.CHOL_ERR_CUDA, L.CHOL_ERR_UNSUPPORTED, L.CHOL_ERR_TIMEOUT, L.CHOL_ERR_WORKSPACE):
        assert L.status_string(st) not in ("success", "unknown status")
    assert L.status_string(12345) == "unknown status"
    assert L.chol_version() >= 100


def test_workspace_bytes(L):
    o = L.opts()
    assert L.chol_workspace_bytes(L.CHOL_CALL_INV, L.CHOL_C64, 1000, 16, 0, o) == 0
    w = L.chol_workspace_bytes(L.CHOL_CALL_INV, L.CHOL_C64, 1000, 16, 1, o)
    assert w >= 1024 + 4 * 1000 and w % 256 == 0
    assert L.chol_workspace_bytes(L.CHOL_CALL_INV, L.CHOL_C64, 0, 16, 1, o) == 0


FAKE = 0x100000  # a non-null pointer value; never dereferenced because validation fails first


@pytest.mark.parametrize("case,expect", [
    (dict(dt=9), "ARG"),
    (dict(batch=-1), "ARG"),
    (dict(max_n=0), "ARG"),
    (dict(max_n=65), "WORKSPACE"),          # blocked path: needs its workspace
    (dict(max_n=65, n=FAKE), "UNSUPPORTED"),  # blocked path: uniform batches only
    (dict(max_n=65, dt=2), "WORKSPACE"),      # blocked path, complex: the real embedding's workspace
    (dict(max_n=65, dt=2, R=2 * FAKE, X=3 * FAKE, ws=FAKE, ws_bytes=1 << 40), "UNSUPPORTED"),  # no complex R
    (dict(max_n=65, dt=3, prec=1, X=3 * FAKE, ws=FAKE, ws_bytes=1 << 40), "UNSUPPORTED"),  # C128: no FP32 modes
    (dict(max_n=65, layout=1), "UNSUPPORTED"),
    (dict(A=None), "ARG"),
    (dict(X=None), "ARG"),
    (dict(layout=2), "ARG"),
    (dict(prec=7), "ARG"),
    (dict(refine=3), "ARG"),
    (dict(flags=0x800), "ARG"),
    (dict(flags=0x300), "ARG"),              # two comparison methods at once
    (dict(flags=0x120), "UNSUPPORTED"),      # a comparison method in the LDL form
    (dict(flags=0x40), "ARG"),               # automatic FP64 pivots keep their redo list in info
    (dict(flags=0x60), "UNSUPPORTED"),       # not with the LDL form
    (dict(prec=1, dt=1), "UNSUPPORTED"),
    (dict(prec=2), "UNSUPPORTED"),
    (dict(prec=3), "UNSUPPORTED"),           # BF16 products: reserved
    (dict(max_n=65, prec=3, ws=FAKE, ws_bytes=1 << 40), "UNSUPPORTED"),
    (dict(n=FAKE), "WORKSPACE"),
    (dict(n=FAKE, ws=FAKE + 8, ws_bytes=1 << 20), "WORKSPACE"),
    (dict(n=FAKE, ws=FAKE, ws_bytes=16), "WORKSPACE"),
])
def test_invalid_arguments_rejected_on_host(L, case, expect):
    a = dict(dt=L.CHOL_F32, batch=10, n=None, off=None, max_n=8, A=FAKE, R=None, X=FAKE, info=None,
             layout=0, prec=0, refine=0, flags=0, ws=None, ws_bytes=0)
    a.update(case)
    o = L.opts(a["prec"], a["refine"], 0, a["layout"], a["flags"])
    st = L.chol_inv_batched(a["dt"], a["batch"], a["n"], a["off"], a["max_n"], a["A"], a["R"], a["X"], a["info"],
                            o, a["ws"], a["ws_bytes"], None)
    assert st == getattr(L, "CHOL_ERR_" + expect)


def test_opts_layout_and_order_set(L):
    # chol_opts_t: five int32 fields, the reserved word, then the 64-bit order set
    assert ctypes.sizeof(L.chol_opts_t) == 32
    assert L.chol_opts_t.orders.offset == 24 and L.chol_opts_t.reserved.offset == 20
    assert L.order_set(None) == 0
    assert L.order_set((4, 8, 16)) == (1 << 3) | (1 << 7) | (1 << 15)
    assert L.order_set([1, 64]) == 1 | (1 << 63)
    for bad in ([0], [65], [-3]):
        with pytest.raises(ValueError):
            L.order_set(bad)
    o = L.opts()
    o.reserved = 1
    st = L.chol_inv_batched(L.CHOL_F32, 10, None, None, 8, FAKE, None, FAKE, None, o, None, 0, None)
    assert st == L.CHOL_ERR_ARG


def test_factor_and_plan_argument_checks(L):
    o = L.opts()
    # the blocked path forms no complex factor
    assert L.chol_factor_batched(L.CHOL_C64, 1, None, None, 65, FAKE, 2 * FAKE, None, o, FAKE, 1 << 40, None) \
        == L.CHOL_ERR_UNSUPPORTED
    assert L.chol_factor_batched(L.CHOL_F64, 3, None, None, 4, FAKE, None, None, o, None, 0, None) == L.CHOL_ERR_ARG
    assert L.chol_factor_batched(L.CHOL_F64, 0, None, None, 4, None, None, None, o, None, 0, None) == L.CHOL_OK
    assert L.chol_plan_inv_create(None, L.CHOL_F32, 1, None, None, 4, FAKE, None, FAKE, None, o, None, 0) \
        == L.CHOL_ERR_ARG
    h = ctypes.c_void_p()
    assert L.chol_plan_inv_create(ctypes.byref(h), L.CHOL_F32, 1, None, None, 99, FAKE, None, FAKE, None, o,
                                  None, 0) == L.CHOL_ERR_UNSUPPORTED
    assert L.chol_plan_launch(None, None) == L.CHOL_ERR_ARG
    assert L.chol_pivot64_redo_count(None, None) == L.CHOL_ERR_ARG
    assert L.chol_plan_destroy(None) == L.CHOL_ERR_ARG
