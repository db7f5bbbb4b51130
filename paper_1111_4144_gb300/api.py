"""PyTorch-facing wrappers of the C ABI (torch supplies device memory and streams).

Every function checks shapes and dtypes, allocates outputs with torch, and
calls one C entry point; all arithmetic happens in libcholinv.so.  Tensors
must be CUDA and contiguous.
"""
from __future__ import annotations

import torch

from . import _lib as L

_DT = {torch.float32: L.CHOL_F32, torch.float64: L.CHOL_F64,
       torch.complex64: L.CHOL_C64, torch.complex128: L.CHOL_C128}

LAYOUT_DENSE = 0
LAYOUT_PACKED = 1


def dtype_code(t: torch.Tensor) -> int:
    try:
        return _DT[t.dtype]
    except KeyError:
        raise ValueError(f"unsupported dtype {t.dtype}") from None


def _need_cuda(*ts):
    for t in ts:
        if t is None:
            continue
        if not t.is_cuda:
            raise ValueError("tensors must be on a CUDA device")
        if not t.is_contiguous():
            raise ValueError("tensors must be contiguous")


def _like(name, t, ref):
    """An output buffer supplied by the caller must match its input in dtype
    and element count (the kernels write as many elements as they read)."""
    if t is None:
        return
    if t.dtype != ref.dtype:
        raise ValueError(f"{name} must have dtype {ref.dtype}, not {t.dtype}")
    if t.numel() != ref.numel():
        raise ValueError(f"{name} must have {ref.numel()} elements, not {t.numel()}")


def _per_matrix(info, off, batch):
    """info (int32) and off (int64) need an entry for every matrix."""
    if info is not None and (info.dtype != torch.int32 or info.numel() < batch):
        raise ValueError(f"info must be int32 with at least {batch} entries")
    if off is not None and off.numel() < batch:
        raise ValueError(f"off must have at least {batch} entries")


def _p(t):
    return None if t is None else t.data_ptr()


def _s(stream):
    return (stream if stream is not None else torch.cuda.current_stream()).cuda_stream


def _geometry(A, n, off, max_n, layout):
    """(batch, max_n) from either a dense (batch, N, N) tensor or a flat buffer + sizes."""
    if n is None and A.dim() == 3:
        if A.shape[1] != A.shape[2]:
            raise ValueError("dense batches must have shape (batch, N, N)")
        if layout != LAYOUT_DENSE:
            raise ValueError("a (batch, N, N) tensor implies the dense layout")
        return A.shape[0], A.shape[1]
    if n is None:
        if max_n is None:
            raise ValueError("a flat buffer needs n (per-matrix sizes) or max_n (uniform size)")
        per = max_n * max_n if layout == LAYOUT_DENSE else max_n * (max_n + 1) // 2
        if A.numel() % per:
            raise ValueError("buffer length is not a multiple of the matrix size")
        return A.numel() // per, max_n
    if n.dtype != torch.int32 or (off is not None and off.dtype != torch.int64):
        raise ValueError("n must be int32 and off int64")
    _need_cuda(n, off)
    batch = n.numel()
    if max_n is None:
        max_n = int(n.max().item()) if batch else 1
    return batch, max(int(max_n), 1)


def workspace(call, dt, batch, max_n, has_sizes, o, device):
    nbytes = L.chol_workspace_bytes(call, dt, batch, max_n, int(has_sizes), o)
    if nbytes == 0:
        return None, 0
    return torch.empty(nbytes, dtype=torch.uint8, device=device), nbytes


def inv(A, n=None, off=None, max_n=None, *, layout=LAYOUT_DENSE, prec=L.CHOL_PREC_NATIVE, refine_steps=0,
        fill_lower=False, want_R=False, flags=0, X=None, R=None, info=None, stream=None, orders=None):
    """Upper half of A^{-1} for every matrix of the batch (Sec. II + Sec. IV.A).

    Returns (X, info) or (X, info, R).  X has A's shape and layout.
    orders: the orders n may hold (an iterable), when known; the call then
    launches kernels for those orders only (chol_opts_t.orders).
    """
    _need_cuda(A, X, R, info)
    dt = dtype_code(A)
    batch, max_n = _geometry(A, n, off, max_n, layout)
    _like("X", X, A)
    _like("R", R, A)
    _per_matrix(info, off, batch)
    o = L.opts(prec, refine_steps, int(fill_lower), layout, flags, orders)
    if X is None:
        X = torch.zeros_like(A)
    if want_R and R is None:
        R = torch.zeros_like(A)
    if info is None:
        info = torch.empty(batch, dtype=torch.int32, device=A.device)
    ws, nbytes = workspace(L.CHOL_CALL_INV, dt, batch, max_n, n is not None, o, A.device)
    st = L.chol_inv_batched(dt, batch, _p(n), _p(off), max_n, _p(A), _p(R), _p(X), _p(info), o,
                            _p(ws), nbytes, _s(stream))
    L.check(st, "chol_inv_batched")
    return (X, info, R) if want_R else (X, info)


class HostInv:
    """Repeated inversions of batches held in host memory (chol_inv_batched_host).

    A_host (and n_host / off_host for per-matrix orders) are CPU tensors,
    pinned for full copy speed; the device workspace for the streaming slots
    is allocated once here.  __call__ enqueues one inversion on `stream` into
    X_host / info_host (CPU tensors) and returns them; synchronise the stream
    before reading them.
    """

    def __init__(self, dtype, batch, max_n, *, sizes=False, layout=LAYOUT_PACKED, prec=L.CHOL_PREC_NATIVE,
                 refine_steps=0, flags=0, device=None):
        self.dt = _DT[dtype]
        self.batch, self.max_n, self.sizes = int(batch), int(max_n), bool(sizes)
        self.o = L.opts(prec, refine_steps, 1 if layout == LAYOUT_DENSE else 0, layout, flags)
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.ws, self.nbytes = workspace(L.CHOL_CALL_INV_HOST, self.dt, self.batch, self.max_n, self.sizes, self.o,
                                         dev)

    def __call__(self, A_host, X_host, n_host=None, off_host=None, info_host=None, stream=None):
        for t in (A_host, X_host, n_host, off_host, info_host):
            if t is not None and (t.is_cuda or not t.is_contiguous()):
                raise ValueError("host tensors must be contiguous CPU tensors")
        if (n_host is not None) != self.sizes:
            raise ValueError("n_host must be given exactly when the plan was made with sizes=True")
        if _DT.get(A_host.dtype) != self.dt:
            raise ValueError(f"A_host has dtype {A_host.dtype}; this HostInv was made for another")
        _like("X_host", X_host, A_host)
        for name, t, dt in (("info_host", info_host, torch.int32), ("n_host", n_host, torch.int32),
                            ("off_host", off_host, torch.int64)):
            if t is not None and (t.dtype != dt or t.numel() < self.batch):
                raise ValueError(f"{name} must be {dt} with at least {self.batch} entries")
        st = L.chol_inv_batched_host(self.dt, self.batch, _p(n_host), _p(off_host), self.max_n, _p(A_host),
                                     _p(X_host), _p(info_host), self.o, _p(self.ws), self.nbytes, _s(stream))
        L.check(st, "chol_inv_batched_host")
        return X_host, info_host


def mmse(H, n=None, m=None, hoff=None, woff=None, max_n=None, max_m=None, *, sigma2=0.0,
         prec=L.CHOL_PREC_NATIVE, refine_steps=0, flags=0, W=None, info=None, stream=None, orders=None):
    """W = (H^* H + sigma2 I)^{-1} H^* for every channel matrix H (with
    sigma2 = 0 and H = D^* square, W^* = D^* (D D^*)^{-1} = D^{-1}, Sec. III.C).

    H: a (batch, M, N) tensor (uniform), or a flat buffer with per-matrix
    n (orders), m (rows), hoff / woff (element offsets of H and W) as device
    tensors, max_n and max_m, and W supplied.  Returns (W, info); W is
    (batch, N, M) for the uniform form."""
    _need_cuda(H, W, info, n, m, hoff, woff)
    dt = dtype_code(H)
    if n is None and m is None and hoff is None and H.dim() == 3:
        batch, max_m, max_n = H.shape
        if W is None:
            W = torch.empty((batch, max_n, max_m), dtype=H.dtype, device=H.device)
    else:
        if n is None or max_n is None or max_m is None or W is None:
            raise ValueError("a flat H needs n, max_n, max_m and W")
        batch = n.numel()
    _like("W", W, W)
    if W.dtype != H.dtype:
        raise ValueError(f"W must have dtype {H.dtype}")
    _per_matrix(info, hoff, batch)
    if info is None:
        info = torch.empty(batch, dtype=torch.int32, device=H.device)
    o = L.opts(prec, refine_steps, 0, LAYOUT_PACKED, flags, orders)
    ws, nbytes = workspace(L.CHOL_CALL_MMSE, dt, batch, max_n, n is not None, o, H.device)
    st = L.chol_mmse_batched(dt, batch, _p(n), _p(m), _p(hoff), _p(woff), int(max_n), int(max_m), _p(H),
                             float(sigma2), _p(W), _p(info), o, _p(ws), nbytes, _s(stream))
    L.check(st, "chol_mmse_batched")
    return W, info


def factor(A, n=None, off=None, max_n=None, *, layout=LAYOUT_DENSE, flags=0, R=None, info=None, stream=None,
           orders=None):
    """Cholesky factor R (Eqs. 3-4).  Returns (R, info)."""
    _need_cuda(A, R, info)
    dt = dtype_code(A)
    batch, max_n = _geometry(A, n, off, max_n, layout)
    _like("R", R, A)
    _per_matrix(info, off, batch)
    o = L.opts(L.CHOL_PREC_NATIVE, 0, 0, layout, flags, orders)
    if R is None:
        R = torch.zeros_like(A)
    if info is None:
        info = torch.empty(batch, dtype=torch.int32, device=A.device)
    ws, nbytes = workspace(L.CHOL_CALL_FACTOR, dt, batch, max_n, n is not None, o, A.device)
    st = L.chol_factor_batched(dt, batch, _p(n), _p(off), max_n, _p(A), _p(R), _p(info), o, _p(ws), nbytes,
                               _s(stream))
    L.check(st, "chol_factor_batched")
    return R, info


def backward(X, G, n=None, off=None, xoff=None, max_n=None, *, layout=LAYOUT_DENSE, upper_param=False, dA=None,
             stream=None):
    """dA = -X (G + G^H)/2 X for every matrix (chol_inv_backward).

    X: forward result (upper half read) in `layout`; G: dense gradient with
    respect to the full X.  Dense (batch, N, N) tensors need no sizes.
    upper_param: return the gradient with respect to the upper triangle
    (the entries the forward call reads) instead of the Hermitian gradient.
    """
    _need_cuda(X, G, dA)
    dt = dtype_code(X)
    if G.dtype != X.dtype:
        raise ValueError("X and G must have the same dtype")
    batch, max_n = _geometry(G, n, off, max_n, LAYOUT_DENSE)
    _like("dA", dA, G)
    if n is None and off is None and xoff is None and layout == LAYOUT_DENSE:
        _like("X", X, G)
    _per_matrix(None, off, batch)
    _per_matrix(None, xoff, batch)
    if dA is None:
        dA = torch.empty_like(G)
    flags = L.CHOL_FLAG_GRAD_UPPER if upper_param else 0
    o = L.opts(L.CHOL_PREC_NATIVE, 0, 0, layout, flags)
    st = L.chol_inv_backward(dt, batch, _p(n), _p(off), _p(xoff), max_n, _p(X), _p(G), _p(dA), o, None, 0,
                             _s(stream))
    L.check(st, "chol_inv_backward")
    return dA


class CholInv(torch.autograd.Function):
    """X = A^{-1} for a dense batch (batch, N, N) of Hermitian positive-definite
    matrices, differentiable.  The forward pass reads the upper triangle of A
    (Sec. II) and returns the full Hermitian X; the backward pass runs the
    adjoint kernel on the saved X (no refactorisation) and returns the
    gradient with respect to the entries the forward pass read."""

    @staticmethod
    def forward(ctx, A, prec=L.CHOL_PREC_NATIVE, refine_steps=0):
        if A.dim() != 3:
            raise ValueError("CholInv expects a (batch, N, N) tensor")
        A = A.contiguous()
        X, info = inv(A, layout=LAYOUT_DENSE, fill_lower=True, prec=prec, refine_steps=refine_steps)
        ctx.save_for_backward(X)
        ctx.mark_non_differentiable(info)
        return X, info

    @staticmethod
    def backward(ctx, gX, ginfo=None):
        (X,) = ctx.saved_tensors
        dA = backward(X, gX.contiguous(), upper_param=True)
        return dA, None, None


def inv_autograd(A, prec=L.CHOL_PREC_NATIVE, refine_steps=0):
    """Differentiable full inverse of a dense batch; returns (X, info)."""
    return CholInv.apply(A, prec, refine_steps)


def autotune(dtype, max_n, *, layout=LAYOUT_PACKED, batch=65536, cache_path=None, stream=None):
    """Time every kernel variant of orders 1..max_n on this GPU and keep the
    fastest (chol_autotune).  Returns {order: chosen variant} for the orders
    that have a choice."""
    dt = _DT[dtype]
    path = cache_path.encode() if cache_path else None
    L.check(L.chol_autotune(dt, int(max_n), int(layout), int(batch), path, _s(stream)), "chol_autotune")
    return {n: L.chol_tune_get(dt, n) for n in range(1, int(max_n) + 1) if L.chol_tune_variants(dt, n) > 1}


def last_device_error(stream=None) -> int:
    return L.chol_last_device_error(_s(stream))


class Plan:
    """A chol_inv_batched call recorded into a CUDA graph; launch() replays it.

    The tensors passed in stay referenced by the plan (the graph holds their
    addresses) until close().
    """

    def __init__(self, A, X, n=None, off=None, max_n=None, *, R=None, info=None, layout=LAYOUT_DENSE,
                 prec=L.CHOL_PREC_NATIVE, refine_steps=0, fill_lower=False, flags=0, timing=False,
                 fixed_orders=False, orders=None):
        """timing: record per-order kernel timing (kernel_ms).  fixed_orders: record
        kernels only for the orders n holds now (CHOL_FLAG_PLAN_ORDERS).  orders:
        the orders n may hold in any replay (chol_opts_t.orders)."""
        import ctypes
        if timing:
            flags |= L.CHOL_FLAG_PLAN_TIMING
        if fixed_orders:
            flags |= L.CHOL_FLAG_PLAN_ORDERS
        _need_cuda(A, X, R, info)
        dt = dtype_code(A)
        batch, max_n = _geometry(A, n, off, max_n, layout)
        _like("X", X, A)
        _like("R", R, A)
        _per_matrix(info, off, batch)
        o = L.opts(prec, refine_steps, int(fill_lower), layout, flags, orders)
        self.info = info if info is not None else torch.empty(batch, dtype=torch.int32, device=A.device)
        self.ws, nbytes = workspace(L.CHOL_CALL_INV, dt, batch, max_n, n is not None, o, A.device)
        self._keep = (A, X, n, off, R, self.info, self.ws)
        h = ctypes.c_void_p()
        st = L.chol_plan_inv_create(ctypes.byref(h), dt, batch, _p(n), _p(off), max_n, _p(A), _p(R), _p(X),
                                    _p(self.info), o, _p(self.ws), nbytes)
        L.check(st, "chol_plan_inv_create")
        self._h = h

    def launch(self, stream=None):
        L.check(L.chol_plan_launch(self._h, _s(stream)), "chol_plan_launch")

    def kernel_ms(self, order):
        """Duration of the order's kernel in the last replay (plan built with timing=True)."""
        import ctypes
        v = ctypes.c_float()
        L.check(L.chol_plan_kernel_ms(self._h, int(order), ctypes.byref(v)), "chol_plan_kernel_ms")
        return float(v.value)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            L.chol_plan_destroy(self._h)
            self._h = None
            self._keep = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
