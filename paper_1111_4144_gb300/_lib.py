"""ctypes binding of libcholinv.so: the C-ABI entry points under their C names.

Argument marshalling only: every function here forwards its arguments to the
library unchanged (pointers and streams as Python ints) and returns the
status code.  The library must exist; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

c_i32 = ctypes.c_int32
c_i64 = ctypes.c_int64
c_size = ctypes.c_size_t
c_vp = ctypes.c_void_p

CHOL_F32, CHOL_F64, CHOL_C64, CHOL_C128 = 0, 1, 2, 3
CHOL_OK, CHOL_ERR_ARG, CHOL_ERR_CUDA, CHOL_ERR_UNSUPPORTED, CHOL_ERR_TIMEOUT, CHOL_ERR_WORKSPACE = 0, -1, -2, -3, -4, -5
CHOL_PREC_NATIVE, CHOL_PREC_FP32_REFINE, CHOL_PREC_TF32_REFINE, CHOL_PREC_BF16_REFINE = 0, 1, 2, 3
CHOL_FLAG_PIVOT64 = 0x1
CHOL_FLAG_GRAD_UPPER = 0x2
CHOL_FLAG_PLAN_TIMING = 0x4
CHOL_FLAG_TF32_SINGLE = 0x8
CHOL_FLAG_PLAN_ORDERS = 0x10
CHOL_FLAG_LDL = 0x20
CHOL_FLAG_PIVOT64_AUTO = 0x40
CHOL_FLAG_RESIDUAL_FP64 = 0x80
CHOL_FLAG_METHOD_ES = 0x100
CHOL_FLAG_METHOD_TMO = 0x200
CHOL_FLAG_SINGLE_LAUNCH = 0x400
CHOL_CALL_FACTOR, CHOL_CALL_INV, CHOL_CALL_BACKWARD, CHOL_CALL_INV_HOST, CHOL_CALL_MMSE = 0, 1, 2, 3, 4
CHOL_BLK_TRAILING_UPDATE, CHOL_BLK_INVERSE_PRODUCT, CHOL_BLK_RESIDUAL, CHOL_BLK_CORRECTION, CHOL_BLK_WHOLE_CALL = \
    0, 1, 2, 3, 4
CHOL_NOALLOC_MAX_BATCH = 1048576


class chol_opts_t(ctypes.Structure):
    _fields_ = [("prec", c_i32), ("refine_steps", c_i32), ("fill_lower", c_i32), ("layout", c_i32),
                ("flags", c_i32), ("reserved", c_i32), ("orders", ctypes.c_uint64)]


# name -> (restype, argtypes); mirrors include/cholinv.h
SIGNATURES = {
    "chol_factor_batched": (c_i32, [c_i32, c_i32, c_vp, c_vp, c_i32, c_vp, c_vp, c_vp,
                                    ctypes.POINTER(chol_opts_t), c_vp, c_size, c_vp]),
    "chol_inv_batched": (c_i32, [c_i32, c_i32, c_vp, c_vp, c_i32, c_vp, c_vp, c_vp, c_vp,
                                 ctypes.POINTER(chol_opts_t), c_vp, c_size, c_vp]),
    "chol_inv_backward": (c_i32, [c_i32, c_i32, c_vp, c_vp, c_vp, c_i32, c_vp, c_vp, c_vp,
                                  ctypes.POINTER(chol_opts_t), c_vp, c_size, c_vp]),
    "chol_inv_batched_noalloc": (c_i32, [c_i32, c_i32, c_vp, c_vp, c_i32, c_vp, c_vp, c_vp, c_vp,
                                         ctypes.POINTER(chol_opts_t), c_vp]),
    "chol_inv_batched_host": (c_i32, [c_i32, c_i32, c_vp, c_vp, c_i32, c_vp, c_vp, c_vp,
                                      ctypes.POINTER(chol_opts_t), c_vp, c_size, c_vp]),
    "chol_mmse_batched": (c_i32, [c_i32, c_i32, c_vp, c_vp, c_vp, c_vp, c_i32, c_i32, c_vp, ctypes.c_double, c_vp,
                                  c_vp, ctypes.POINTER(chol_opts_t), c_vp, c_size, c_vp]),
    "chol_workspace_bytes": (c_size, [c_i32, c_i32, c_i32, c_i32, c_i32, ctypes.POINTER(chol_opts_t)]),
    "chol_status_string": (ctypes.c_char_p, [c_i32]),
    "chol_last_device_error": (c_i32, [c_vp]),
    "chol_pivot64_redo_count": (c_i32, [c_vp, ctypes.POINTER(c_i64)]),
    "chol_blocked_timing": (c_i32, [c_i32]),
    "chol_blocked_timing_read": (c_i32, [c_i32, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(c_i32)]),
    "chol_version": (c_i32, []),
    "chol_plan_inv_create": (c_i32, [ctypes.POINTER(c_vp), c_i32, c_i32, c_vp, c_vp, c_i32, c_vp, c_vp, c_vp,
                                     c_vp, ctypes.POINTER(chol_opts_t), c_vp, c_size]),
    "chol_plan_launch": (c_i32, [c_vp, c_vp]),
    "chol_plan_destroy": (c_i32, [c_vp]),
    "chol_plan_kernel_ms": (c_i32, [c_vp, c_i32, ctypes.POINTER(ctypes.c_float)]),
    "chol_autotune": (c_i32, [c_i32, c_i32, c_i32, c_i32, ctypes.c_char_p, c_vp]),
    "chol_tune_load": (c_i32, [ctypes.c_char_p]),
    "chol_tune_variants": (c_i32, [c_i32, c_i32]),
    "chol_tune_get": (c_i32, [c_i32, c_i32]),
    "chol_tune_set": (c_i32, [c_i32, c_i32, c_i32]),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libcholinv.so (building it first if asked and it is missing)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if build_if_missing:
                path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library {path} is missing; run paper_1111_4144_gb300/build.py")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def status_string(status: int) -> str:
    return load().chol_status_string(status).decode()


class CholError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {status_string(status)} ({status})")
        self.status = status


def check(status: int, what: str) -> None:
    if status != CHOL_OK:
        raise CholError(status, what)


def order_set(orders) -> int:
    """chol_opts_t.orders for an iterable of matrix orders (1..64); 0 for None."""
    if orders is None:
        return 0
    m = 0
    for c in orders:
        c = int(c)
        if not 1 <= c <= 64:
            raise ValueError(f"order {c} outside 1..64")
        m |= 1 << (c - 1)
    return m


def opts(prec=CHOL_PREC_NATIVE, refine_steps=0, fill_lower=0, layout=0, flags=0, orders=None) -> chol_opts_t:
    return chol_opts_t(int(prec), int(refine_steps), int(fill_lower), int(layout), int(flags), 0, order_set(orders))


# raw entry points, same names as the C ABI
def chol_factor_batched(*args):
    return load().chol_factor_batched(*args)


def chol_inv_batched(*args):
    return load().chol_inv_batched(*args)


def chol_inv_backward(*args):
    return load().chol_inv_backward(*args)


def chol_inv_batched_noalloc(*args):
    return load().chol_inv_batched_noalloc(*args)


def chol_inv_batched_host(*args):
    return load().chol_inv_batched_host(*args)


def chol_mmse_batched(*args):
    return load().chol_mmse_batched(*args)


def chol_workspace_bytes(*args):
    return load().chol_workspace_bytes(*args)


def chol_status_string(*args):
    return load().chol_status_string(*args)


def chol_last_device_error(*args):
    return load().chol_last_device_error(*args)


def chol_pivot64_redo_count(*args):
    return load().chol_pivot64_redo_count(*args)


def chol_blocked_timing(*args):
    return load().chol_blocked_timing(*args)


def chol_blocked_timing_read(*args):
    return load().chol_blocked_timing_read(*args)


def chol_version():
    return load().chol_version()


def chol_plan_inv_create(*args):
    return load().chol_plan_inv_create(*args)


def chol_plan_launch(*args):
    return load().chol_plan_launch(*args)


def chol_plan_destroy(*args):
    return load().chol_plan_destroy(*args)


def chol_plan_kernel_ms(*args):
    return load().chol_plan_kernel_ms(*args)


def chol_autotune(*args):
    return load().chol_autotune(*args)


def chol_tune_load(*args):
    return load().chol_tune_load(*args)


def chol_tune_variants(*args):
    return load().chol_tune_variants(*args)


def chol_tune_get(*args):
    return load().chol_tune_get(*args)


def chol_tune_set(*args):
    return load().chol_tune_set(*args)
