"""CPU FP64 oracle for the Cholesky factor + direct inverse of arXiv 1111.4144.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg import this package.  The GPU library never calls it, and it
shares no code with the GPU library.  The arithmetic lives in ``oracle.c``
(plain C loops, IEEE binary64, no fused multiply-add); this module compiles it
with gcc and wraps it with ctypes and numpy.

Function map (paper passages are cited in ``oracle.c``):
  chol(A)               Sec. II, Eqs. 3-4        -> (R, info)
  inv_rows(R)           Sec. IV.A, Eqs. 20-24    -> upper X (rows N..1)
  inv_cols(R)           Sec. IV.A                -> upper X (columns N..1)
  es(R), tmo(R)         Sec. III.A / III.B       -> upper X, multiply count
  ldl(A), ldl_inv(R, d) Sec. II.A / IV.B         -> LDL factor / inverse
  gj(A)                 long-double Gauss-Jordan -> full inverse (independent)
  grad(X, G)            dA = -X (G+G^H)/2 X
  inv_batch(...)        batched driver over per-matrix sizes and offsets
  chol_mt, inv_rows_mt  chol / inv_rows for one large real matrix on several threads (same bits)
  solve_cols(R, cols)   chosen columns of A^{-1} by Eq. 15's two triangular solves (every row)
  nonhermitian_inverse  Sec. III.C: D^{-1} = D^* (D D^*)^{-1}
  mmse_filter(H, s2)    (H^* H + s2 I)^{-1} H^*, the consumer of the MIMO matrices
The fixed-point emulation of the methods (Sec. IV.C) is ``fixedpoint.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIBDIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

_P = ctypes.POINTER
_d = _P(ctypes.c_double)
_ll = _P(ctypes.c_longlong)
_i32 = _P(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/lib/liboracle.so (gcc, -ffp-contract=off)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-pthread", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            for name in ("orc_chol_d", "orc_chol_z"):
                f = getattr(lib, name); f.restype = ctypes.c_int; f.argtypes = [ctypes.c_int, _d, _d, _ll]
            for name in ("orc_inv_rows_d", "orc_inv_rows_z", "orc_inv_cols_d", "orc_inv_cols_z",
                         "orc_es_d", "orc_es_z"):
                f = getattr(lib, name); f.restype = None; f.argtypes = [ctypes.c_int, _d, _d, _ll]
            for name in ("orc_tmo_d", "orc_tmo_z"):
                f = getattr(lib, name); f.restype = None; f.argtypes = [ctypes.c_int, _d, _d, ctypes.c_int, _ll]
            for name in ("orc_ldl_d", "orc_ldl_z"):
                f = getattr(lib, name); f.restype = ctypes.c_int; f.argtypes = [ctypes.c_int, _d, _d, _d, _ll]
            for name in ("orc_ldl_inv_d", "orc_ldl_inv_z"):
                f = getattr(lib, name); f.restype = None; f.argtypes = [ctypes.c_int, _d, _d, _d, _ll]
            for name in ("orc_gj_ld", "orc_gj_lz"):
                f = getattr(lib, name); f.restype = ctypes.c_int; f.argtypes = [ctypes.c_int, _d, _d]
            for name in ("orc_grad_d", "orc_grad_z"):
                f = getattr(lib, name); f.restype = None; f.argtypes = [ctypes.c_int, _d, _d, _d]
            lib.orc_chol_mt_d.restype = ctypes.c_int
            lib.orc_chol_mt_d.argtypes = [ctypes.c_int, _d, _d, ctypes.c_int]
            lib.orc_inv_rows_mt_d.restype = None
            lib.orc_inv_rows_mt_d.argtypes = [ctypes.c_int, _d, _d, ctypes.c_int]
            lib.orc_solve_cols_d.restype = None
            lib.orc_solve_cols_d.argtypes = [ctypes.c_int, _d, ctypes.c_int, _i32, _d, ctypes.c_int]
            lib.orc_inv_batch.restype = ctypes.c_int
            lib.orc_inv_batch.argtypes = [ctypes.c_int, ctypes.c_longlong, _i32, _ll, ctypes.c_int, ctypes.c_int,
                                          _d, _d, _d, _i32, ctypes.c_int]
            _lib = lib
    return _lib


def _as_dense(A):
    A = np.asarray(A)
    cplx = np.iscomplexobj(A)
    A = np.ascontiguousarray(A, dtype=np.complex128 if cplx else np.float64)
    return A, cplx


def _ptr(a):
    return a.ctypes.data_as(_d)


class _Count:
    def __init__(self):
        self.c = ctypes.c_longlong(0)

    @property
    def ref(self):
        return ctypes.byref(self.c)

    @property
    def value(self):
        return int(self.c.value)


def chol(A, count=False):
    """Cholesky A = R^* R (Eqs. 3-4).  Returns (R, info[, multiplies])."""
    lib = _load()
    A, cplx = _as_dense(A)
    n = A.shape[0]
    R = np.zeros_like(A)
    c = _Count()
    info = (lib.orc_chol_z if cplx else lib.orc_chol_d)(n, _ptr(A), _ptr(R), c.ref)
    return (R, info, c.value) if count else (R, info)


def _inv_from_R(fn_d, fn_z, R, count):
    lib = _load()
    R, cplx = _as_dense(R)
    n = R.shape[0]
    X = np.zeros_like(R)
    c = _Count()
    getattr(lib, fn_z if cplx else fn_d)(n, _ptr(R), _ptr(X), c.ref)
    return (X, c.value) if count else X


def inv_rows(R, count=False):
    """Proposed inverse (Eqs. 20-24), rows N..1; upper half of X, lower zero."""
    return _inv_from_R("orc_inv_rows_d", "orc_inv_rows_z", R, count)


def inv_cols(R, count=False):
    """Proposed inverse (Eqs. 20-24), columns N..1; upper half of X, lower zero."""
    return _inv_from_R("orc_inv_cols_d", "orc_inv_cols_z", R, count)


def es(R, count=False):
    """Existing method 'Equation Solving' (Eq. 15); upper half of X."""
    return _inv_from_R("orc_es_d", "orc_es_z", R, count)


def tmo(R, exploit=False, count=False):
    """Existing method 'Triangular Matrix Operations' (Eqs. 16-19); upper half of X."""
    lib = _load()
    R, cplx = _as_dense(R)
    n = R.shape[0]
    X = np.zeros_like(R)
    c = _Count()
    (lib.orc_tmo_z if cplx else lib.orc_tmo_d)(n, _ptr(R), _ptr(X), int(bool(exploit)), c.ref)
    return (X, c.value) if count else X


def ldl(A, count=False):
    """LDL decomposition A = R^* D R (Eqs. 10-11).  Returns (R, d, info[, mults])."""
    lib = _load()
    A, cplx = _as_dense(A)
    n = A.shape[0]
    R = np.zeros_like(A)
    d = np.zeros(n, dtype=np.float64)
    c = _Count()
    info = (lib.orc_ldl_z if cplx else lib.orc_ldl_d)(n, _ptr(A), _ptr(R), _ptr(d), c.ref)
    return (R, d, info, c.value) if count else (R, d, info)


def ldl_inv(R, d, count=False):
    """Proposed inverse through LDL (Eqs. 25-29); upper half of X."""
    lib = _load()
    R, cplx = _as_dense(R)
    d = np.ascontiguousarray(d, dtype=np.float64)
    n = R.shape[0]
    X = np.zeros_like(R)
    c = _Count()
    (lib.orc_ldl_inv_z if cplx else lib.orc_ldl_inv_d)(n, _ptr(R), _ptr(d), _ptr(X), c.ref)
    return (X, c.value) if count else X


def gj(A):
    """Gauss-Jordan inverse in long double of the Hermitian matrix whose upper triangle is A's."""
    lib = _load()
    A, cplx = _as_dense(A)
    n = A.shape[0]
    X = np.zeros_like(A)
    rc = (lib.orc_gj_lz if cplx else lib.orc_gj_ld)(n, _ptr(A), _ptr(X))
    if rc:
        raise np.linalg.LinAlgError("singular matrix in Gauss-Jordan")
    return X


def grad(X, G):
    """dA = -X S X with S = (G + G^H)/2; X full Hermitian, G full."""
    lib = _load()
    X, cplx = _as_dense(X)
    G = np.ascontiguousarray(G, dtype=X.dtype)
    n = X.shape[0]
    dA = np.zeros_like(X)
    (lib.orc_grad_z if cplx else lib.orc_grad_d)(n, _ptr(X), _ptr(G), _ptr(dA))
    return dA


def chol_mt(A, nthreads=None):
    """chol(A) for one real matrix with the entries of each row split over
    threads; the same operations in the same order, so the same bits."""
    lib = _load()
    A = np.ascontiguousarray(A, dtype=np.float64)
    n = A.shape[0]
    R = np.zeros_like(A)
    info = lib.orc_chol_mt_d(n, _ptr(A), _ptr(R), int(nthreads or os.cpu_count() or 1))
    return R, info


def inv_rows_mt(R, nthreads=None):
    """inv_rows(R) for one real matrix, threaded like chol_mt (the same bits)."""
    lib = _load()
    R = np.ascontiguousarray(R, dtype=np.float64)
    n = R.shape[0]
    X = np.zeros_like(R)
    lib.orc_inv_rows_mt_d(n, _ptr(R), _ptr(X), int(nthreads or os.cpu_count() or 1))
    return X


def solve_cols(R, cols, nthreads=None):
    """Columns `cols` of A^{-1} (A = R^T R, real) by the two triangular solves
    of Eq. 15, R^T y = e_j then R x = y, each column on its own (every row,
    no values taken from other columns).  Returns an array [len(cols), n]
    whose row c is column cols[c] of A^{-1}."""
    lib = _load()
    R = np.ascontiguousarray(R, dtype=np.float64)
    n = R.shape[0]
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    Xc = np.zeros((len(cols), n), dtype=np.float64)
    lib.orc_solve_cols_d(n, _ptr(R), len(cols), cols.ctypes.data_as(_i32), _ptr(Xc),
                         int(nthreads or os.cpu_count() or 1))
    return Xc


def inverse(A):
    """Proposed method end to end: Cholesky then the direct inverse.  Returns (R, X_upper, info)."""
    R, info = chol(A)
    if info:
        return R, None, info
    return R, inv_rows(R), info


def full_hermitian(Xu):
    """Mirror an upper-half matrix into the full Hermitian one (x_ji = conj(x_ij))."""
    Xu = np.asarray(Xu)
    U = np.triu(Xu)
    L = np.conj(np.triu(Xu, 1)).T
    return U + L


def nonhermitian_inverse(D):
    """Sec. III.C: the inverse of an arbitrary square D through the Hermitian
    A = D D^* (product by numpy), A^{-1} by the proposed method (Cholesky,
    Eqs. 3-4, then Sec. IV.A), and D^{-1} = D^* A^{-1}.  Returns (D^{-1}, info);
    info != 0 (D singular to working precision) gives None."""
    D = np.asarray(D)
    cplx = np.iscomplexobj(D)
    D = D.astype(np.complex128 if cplx else np.float64)
    A = D @ np.conj(D).T
    _, Xu, info = inverse(A)
    if info:
        return None, info
    return np.conj(D).T @ full_hermitian(Xu), 0


def mmse_filter(H, sigma2):
    """W = (H^* H + sigma2 I)^{-1} H^* for an M x N channel H (M >= N): the
    Hermitian inverse by the proposed method, then one product (numpy).  The
    matrices of the MIMO workload are these A = H^* H + sigma2 I; W is their
    usual consumer (not a formula of the paper).  Returns (W, info)."""
    H = np.asarray(H)
    cplx = np.iscomplexobj(H)
    H = H.astype(np.complex128 if cplx else np.float64)
    N = H.shape[1]
    A = np.conj(H).T @ H + sigma2 * np.eye(N)
    _, Xu, info = inverse(A)
    if info:
        return None, info
    return full_hermitian(Xu) @ np.conj(H).T, 0


def inv_batch(A_flat, n, off, layout, cplx, want_R=False, fill_lower=False, nthreads=None):
    """Batched proposed inverse over a flat buffer.

    A_flat: float64 (complex: interleaved pairs as a complex128 array) holding every
    matrix at element offset off[b] with order n[b]; layout 0 dense, 1 packed upper.
    Returns (R_flat or None, X_flat, info).  X_flat/R_flat are zero where not written.
    """
    lib = _load()
    A_flat = np.ascontiguousarray(A_flat, dtype=np.complex128 if cplx else np.float64)
    n = np.ascontiguousarray(n, dtype=np.int32)
    off = np.ascontiguousarray(off, dtype=np.int64)
    batch = int(n.shape[0])
    X = np.zeros_like(A_flat)
    R = np.zeros_like(A_flat) if want_R else None
    info = np.zeros(batch, dtype=np.int32)
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    lib.orc_inv_batch(int(cplx), batch, n.ctypes.data_as(_i32), off.ctypes.data_as(_ll), int(layout),
                      int(bool(fill_lower)), _ptr(A_flat), _ptr(R) if R is not None else None, _ptr(X),
                      info.ctypes.data_as(_i32), int(nthreads))
    return R, X, info


# ---------------------------------------------------------------------------
# Multiply counts in closed form, as the paper states them (Table 1) and as the
# counting convention above gives them exactly.
# ---------------------------------------------------------------------------
def count_closed_form(n: int) -> dict:
    """Exact multiply counts of each method under the accounting of oracle.c."""
    chol_ = (n ** 3 - n) // 6
    return {
        "cholesky": chol_,
        "proposed_solve": (n ** 3 - n) // 3,
        "proposed": (n ** 3 - n) // 2,
        "es": chol_ + 2 * ((n ** 3 - n) // 3),
        "tmo": chol_ + (n ** 3 - n) // 3 + n * (n + 1) * (n + 2) // 6,
        "tmo_exploit": chol_ + (n ** 3 - n) // 6 + n * (n + 1) * (n + 2) // 6,
    }
