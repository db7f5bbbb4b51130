"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
on a seeded batch, run the oracle on the same (rounded) inputs, and measure
per-matrix relative Frobenius errors over the upper triangle."""
from __future__ import annotations

import numpy as np

from paper_1111_4144_gb300 import workloads as wl

NP_OF = {"f32": np.float32, "f64": np.float64, "c64": np.complex64, "c128": np.complex128}
WIDE_OF = {"f32": np.float64, "f64": np.float64, "c64": np.complex128, "c128": np.complex128}

U32 = 2.0 ** -24
TOL64 = 1e-11


def tol32(kappa):
    """FP32 tolerance: relative Frobenius error <= max(1e-7 * kappa, 2.4e-7)."""
    return np.maximum(1e-7 * np.asarray(kappa), 2.4e-7)


def check_errors(tag, b, A_wide, err, what):
    """Assert every matrix's error is within the tolerance of its precision."""
    if tag in ("f64", "c128"):
        tol = np.full(b.batch, TOL64)
    else:
        tol = tol32(kappas(b, A_wide))
    bad = np.nonzero(~(err <= tol))[0]
    assert bad.size == 0, f"{what}: {bad.size} of {b.batch} matrices over tolerance; worst ratio " \
                          f"{np.max(err / tol):.3g} at matrix {bad[0]} (N={b.n[bad[0]]})"


def torch_dtype(tag):
    import torch
    return {"f32": torch.float32, "f64": torch.float64, "c64": torch.complex64, "c128": torch.complex128}[tag]


def cast_batch(b: wl.Batch, tag):
    """Round the batch to the working precision, then widen back for the oracle."""
    A = b.A.astype(NP_OF[tag])
    return A, A.astype(WIDE_OF[tag])


def kappas(b: wl.Batch, A_wide):
    """2-norm condition numbers of the (rounded) matrices."""
    out = np.zeros(b.batch)
    bb = wl.Batch(A_wide, b.n, b.off, b.layout)
    for k in range(b.batch):
        M = bb.matrix(k)
        M = np.triu(M) + np.conj(np.triu(M, 1)).T
        if M.shape[0] == 0:
            out[k] = 1.0
            continue
        ev = np.linalg.eigvalsh(M)
        out[k] = ev[-1] / ev[0] if ev[0] > 0 else np.inf
    return out


def upper_errors(b: wl.Batch, got_flat, ref_flat):
    """Per-matrix ||upper(got - ref)||_F / ||upper(ref)||_F."""
    g = wl.Batch(np.asarray(got_flat).astype(np.complex128 if np.iscomplexobj(got_flat) else np.float64),
                 b.n, b.off, b.layout)
    r = wl.Batch(ref_flat, b.n, b.off, b.layout)
    err = np.zeros(b.batch)
    for k in range(b.batch):
        G = g.matrix(k)
        Rm = r.matrix(k)
        den = np.linalg.norm(Rm)
        err[k] = np.linalg.norm(G - Rm) / den if den > 0 else np.linalg.norm(G - Rm)
    return err


def run_inv(b: wl.Batch, tag, *, mixed, want_R=False, fill_lower=False, plan=False, stream=None, **kw):
    """Run chol_inv_batched on batch b; returns (X_flat np, info np, R_flat np or None)."""
    import torch
    from paper_1111_4144_gb300 import api
    A_np, _ = cast_batch(b, tag)
    dev = torch.device("cuda", 0)
    A = torch.from_numpy(A_np).to(dev)
    n = torch.from_numpy(b.n).to(dev) if mixed else None
    off = torch.from_numpy(b.off).to(dev) if mixed else None
    max_n = int(b.n.max()) if b.batch else 1
    if plan:
        X = torch.zeros_like(A)
        R = torch.zeros_like(A) if want_R else None
        p = api.Plan(A, X, n, off, max_n, R=R, layout=b.layout, fill_lower=fill_lower, **kw)
        p.launch()
        torch.cuda.synchronize()
        out = (X.cpu().numpy(), p.info.cpu().numpy(), None if R is None else R.cpu().numpy())
        p.close()
        return out
    res = api.inv(A, n, off, max_n, layout=b.layout, want_R=want_R, fill_lower=fill_lower, **kw)
    torch.cuda.synchronize()
    X, info = res[0], res[1]
    R = res[2] if want_R else None
    return X.cpu().numpy(), info.cpu().numpy(), None if R is None else R.cpu().numpy()


def oracle_inv(orc, b: wl.Batch, tag, fill_lower=False):
    _, A_wide = cast_batch(b, tag)
    R, X, info = orc.inv_batch(A_wide, b.n, b.off, b.layout, np.iscomplexobj(A_wide), want_R=True,
                               fill_lower=fill_lower)
    return R, X, info, A_wide


def sub_batch(b: wl.Batch, idx, flat=None):
    """Matrices idx of batch b (elements taken from `flat`, default b.A),
    laid out back to back in b's layout, as a new Batch."""
    flat = b.A if flat is None else np.asarray(flat)
    idx = np.asarray(idx, dtype=np.int64)
    n = b.n[idx].astype(np.int32)
    off, total = wl.layout_offsets(n, b.layout)
    per = wl.tri(n.astype(np.int64)) if b.layout == wl.LAYOUT_PACKED else n.astype(np.int64) ** 2
    out = np.zeros(total, dtype=flat.dtype)
    for k, src in enumerate(b.off[idx]):
        out[off[k]:off[k] + per[k]] = flat[src:src + per[k]]
    return wl.Batch(out, n, off, b.layout)


def diagonal_positions(b: wl.Batch):
    """Flat element positions of every diagonal entry of every matrix of b."""
    n = b.n.astype(np.int64)
    owner = np.repeat(np.arange(b.batch), n)
    i = np.arange(int(n.sum()), dtype=np.int64) - np.repeat(np.cumsum(n) - n, n)
    N = n[owner]
    if b.layout == wl.LAYOUT_PACKED:
        return b.off[owner] + i * N - i * (i - 1) // 2
    return b.off[owner] + i * (N + 1)
