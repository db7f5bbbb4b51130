"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random numbers and lays matrices out in memory; it holds
none of the factorisation or inversion arithmetic.  Both the GPU tests and the
CPU oracle take their inputs from here, so the two sides always see the same
matrices.  Every generator works in float64 / complex128 on the host and the
caller casts to the working precision.

Layouts (shared with the C-ABI): matrix b has order n[b] and starts at element
off[b] of a flat buffer.  Layout 0 = dense row-major n*n; layout 1 = upper
triangle packed row by row (row i holds columns i..n-1), n(n+1)/2 elements.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

LAYOUT_DENSE = 0
LAYOUT_PACKED = 1


def tri(n):
    """Number of elements in the upper triangle of an n x n matrix."""
    return n * (n + 1) // 2


@dataclass
class Batch:
    """A flat batch of Hermitian matrices plus their sizes and offsets."""
    A: np.ndarray            # flat, float64 or complex128
    n: np.ndarray            # int32 [batch]
    off: np.ndarray          # int64 [batch]
    layout: int
    kappa: np.ndarray | None = None   # per-matrix 2-norm condition number, when the generator fixes it
    meta: dict = field(default_factory=dict)

    @property
    def batch(self):
        return int(self.n.shape[0])

    @property
    def is_complex(self):
        return np.iscomplexobj(self.A)

    def matrix(self, b):
        """Dense upper-triangular view (lower part zero) of matrix b, as a new array."""
        n = int(self.n[b]); o = int(self.off[b])
        M = np.zeros((n, n), dtype=self.A.dtype)
        iu = np.triu_indices(n)
        if self.layout == LAYOUT_PACKED:
            M[iu] = self.A[o:o + tri(n)]
        else:
            M[iu] = self.A[o:o + n * n].reshape(n, n)[iu]
        return M

    def sizes_offsets(self):
        return self.n, self.off


def layout_offsets(n, layout):
    """Contiguous element offsets for sizes n in the given layout."""
    n = np.asarray(n, dtype=np.int64)
    per = tri(n) if layout == LAYOUT_PACKED else n * n
    off = np.zeros(n.shape[0], dtype=np.int64)
    if n.shape[0] > 1:
        off[1:] = np.cumsum(per)[:-1]
    total = int(per.sum()) if n.shape[0] else 0
    return off, total


def pack(dense_by_index, n, layout, dtype):
    """Lay out full matrices (a dict size -> (indices, stack)) into one flat buffer."""
    off, total = layout_offsets(n, layout)
    A = np.zeros(total, dtype=dtype)
    for N, (idx, stack) in dense_by_index.items():
        if len(idx) == 0:
            continue
        if layout == LAYOUT_PACKED:
            iu = np.triu_indices(N)
            vals = stack[:, iu[0], iu[1]]                       # [m, T]
            pos = off[idx][:, None] + np.arange(tri(N))[None, :]
        else:
            vals = stack.reshape(len(idx), N * N)
            pos = off[idx][:, None] + np.arange(N * N)[None, :]
        A[pos] = vals
    return A, off


def _group(n):
    out = {}
    for N in np.unique(n):
        out[int(N)] = np.nonzero(n == N)[0]
    return out


def _haar_orthogonal(rng, m, N):
    """Q from the Householder QR of an N x N Gaussian, R's diagonal made positive."""
    G = rng.standard_normal((m, N, N))
    Q, Rq = np.linalg.qr(G)
    s = np.sign(np.diagonal(Rq, axis1=1, axis2=2)).copy()
    s[s == 0] = 1.0
    return Q * s[:, None, :]


def spd_gram_shift(batch, N, shift, seed, layout=LAYOUT_DENSE):
    """A = B B^T + shift*I with B iid N(0,1), N x N (real)."""
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((batch, N, N))
    A = B @ np.transpose(B, (0, 2, 1)) + shift * np.eye(N)
    A = 0.5 * (A + np.transpose(A, (0, 2, 1)))
    n = np.full(batch, N, dtype=np.int32)
    flat, off = pack({N: (np.arange(batch), A)}, n, layout, np.float64)
    return Batch(flat, n, off, layout, meta={"kind": "gram_shift", "N": N, "shift": shift, "seed": seed})


def mimo_covariance(batch, sizes=(4, 8, 16), sigma2=0.1, seed=1001, layout=LAYOUT_PACKED, chunk=65536,
                    shuffle=True):
    """A = H^H H + sigma2*I, H a 2N x N matrix of iid CN(0,1) entries (complex).

    The batch holds the sizes in equal shares (the first batch % len(sizes)
    sizes get one more), in an order shuffled with the seed.
    """
    rng = np.random.default_rng(seed)
    k = len(sizes)
    counts = [batch // k + (1 if i < batch % k else 0) for i in range(k)]
    n = np.concatenate([np.full(c, s, dtype=np.int32) for s, c in zip(sizes, counts)])
    if shuffle:
        n = n[rng.permutation(batch)]
    groups = _group(n)
    dense = {}
    for N, idx in groups.items():
        stacks = []
        for s in range(0, len(idx), chunk):
            m = min(chunk, len(idx) - s)
            H = (rng.standard_normal((m, 2 * N, N)) + 1j * rng.standard_normal((m, 2 * N, N))) * np.sqrt(0.5)
            A = np.conj(np.transpose(H, (0, 2, 1))) @ H
            A += sigma2 * np.eye(N)
            stacks.append(A)
        dense[N] = (idx, np.concatenate(stacks))
    flat, off = pack(dense, n, layout, np.complex128)
    return Batch(flat, n, off, layout, meta={"kind": "mimo", "sizes": list(sizes), "sigma2": sigma2, "seed": seed})


def qr_spectrum(batch, n_of, lam_of, seed, layout=LAYOUT_DENSE, chunk=8192):
    """A = Q diag(lam) Q^T, Q Haar-orthogonal from Householder QR of a Gaussian.

    n_of(rng, batch) -> int32 sizes; lam_of(rng, m, N) -> [m, N] eigenvalues.
    The result is symmetrised in float64.  kappa holds max(lam)/min(lam).
    """
    rng = np.random.default_rng(seed)
    n = np.asarray(n_of(rng, batch), dtype=np.int32)
    kappa = np.zeros(batch)
    dense = {}
    for N, idx in _group(n).items():
        stacks = []
        for s in range(0, len(idx), chunk):
            m = min(chunk, len(idx) - s)
            Q = _haar_orthogonal(rng, m, N)
            lam = np.asarray(lam_of(rng, m, N), dtype=np.float64)
            A = (Q * lam[:, None, :]) @ np.transpose(Q, (0, 2, 1))
            A = 0.5 * (A + np.transpose(A, (0, 2, 1)))
            stacks.append(A)
            kappa[idx[s:s + m]] = lam.max(axis=1) / lam.min(axis=1)
        dense[N] = (idx, np.concatenate(stacks))
    flat, off = pack(dense, n, layout, np.float64)
    return Batch(flat, n, off, layout, kappa=kappa, meta={"kind": "qr_spectrum", "seed": seed})


def uneven_loguniform(batch, nmin=2, nmax=64, decades=3.0, seed=1002, layout=LAYOUT_DENSE):
    """N ~ U{nmin..nmax}; lam_i = 10^U(0, decades) (log-uniform in [1, 10^decades])."""
    return qr_spectrum(batch,
                       lambda rng, b: rng.integers(nmin, nmax + 1, size=b),
                       lambda rng, m, N: 10.0 ** rng.uniform(0.0, decades, size=(m, N)),
                       seed, layout)


def fixed_kappa(batch, N, kappa, seed=1003, layout=LAYOUT_DENSE):
    """lam_1 = 1, lam_N = kappa, the rest log-uniform in between (kappa exact)."""
    def lam(rng, m, NN):
        L = 10.0 ** rng.uniform(0.0, np.log10(kappa), size=(m, NN))
        L[:, 0] = 1.0
        L[:, -1] = kappa
        return L
    return qr_spectrum(batch, lambda rng, b: np.full(b, N), lam, seed, layout)


def log_spaced(N, decades=4.0, seed=1004, layout=LAYOUT_DENSE):
    """A single matrix with lam_i = 10^(decades*(i-1)/(N-1))."""
    return qr_spectrum(1, lambda rng, b: np.full(b, N),
                       lambda rng, m, NN: np.tile(10.0 ** (decades * np.arange(NN) / max(NN - 1, 1)), (m, 1)),
                       seed, layout, chunk=1)


def gaussian(shape, seed, complex_=False):
    """iid N(0,1) (complex: CN(0,1)) array, e.g. the weights W of a loss sum(W o X)."""
    rng = np.random.default_rng(seed)
    if complex_:
        return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * np.sqrt(0.5)
    return rng.standard_normal(shape)


def bordered_cancellation(batch, N, ratio=16.0, seed=1005, layout=LAYOUT_PACKED, complex_=False):
    """Hermitian PD matrices whose last pivot cancels: A = D [[I, c], [c^*, d]] D.

    c (N-1 entries, iid N(0,1), complex: CN(0,1)) is drawn exactly
    representable in FP32 (each part rounded to float32), d = |c|^2 (1 + ratio
    2^-24) in float64, and D = diag(2^e_i) with e_i uniform on {-2..2} (an
    exact scaling).  The Schur complement of the identity block,
    d - |c|^2 (times the scaling), is about `ratio` FP32 ulps of d: the
    argument of the last pivot is a difference of two nearly equal numbers,
    while every other pivot and every entry above it is exact in FP32.
    The caller casts to the working precision (only d is rounded then).
    """
    rng = np.random.default_rng(seed)
    dt = np.complex128 if complex_ else np.float64
    dense = np.zeros((batch, N, N), dtype=dt)
    for b in range(batch):
        c = rng.standard_normal(N - 1)
        if complex_:
            c = (c + 1j * rng.standard_normal(N - 1)) * np.sqrt(0.5)
            c = c.real.astype(np.float32).astype(np.float64) + 1j * c.imag.astype(np.float32).astype(np.float64)
        else:
            c = c.astype(np.float32).astype(np.float64)
        M = np.eye(N, dtype=dt)
        M[:N - 1, N - 1] = c
        M[N - 1, :N - 1] = np.conj(c)
        s = float(np.sum(np.abs(c) ** 2))
        M[N - 1, N - 1] = s * (1.0 + ratio * 2.0 ** -24)
        e = 2.0 ** rng.integers(-2, 3, size=N)
        dense[b] = (e[:, None] * M) * e[None, :]
    n = np.full(batch, N, dtype=np.int32)
    flat, off = pack({N: (np.arange(batch), dense)}, n, layout, dt)
    return Batch(flat, n, off, layout, meta={"kind": "bordered_cancellation", "N": N, "ratio": ratio, "seed": seed})


def rotated_log_spaced_torch(N, decades=4.0, seed=1004, reflections=8, device="cuda"):
    """A = H_r ... H_1 diag(lam) H_1 ... H_r, lam_i = 10^(decades (i-1)/(N-1)),
    H_k = I - 2 v_k v_k^T with v_k a normalised Gaussian vector (torch's
    generator on `device`, seeded): the spectrum of log_spaced without a QR
    factorisation, for orders too large to factor on the host (another,
    non-Haar eigenbasis).  Each reflection is applied as the rank-2 update
    A <- A - 2 v w^T - 2 w v^T + 4 (v^T w) v v^T, w = A v.  Returns the float64
    N x N tensor on `device`, symmetrised."""
    import torch
    g = torch.Generator(device=device).manual_seed(seed)
    lam = 10.0 ** (decades * torch.arange(N, dtype=torch.float64, device=device) / max(N - 1, 1))
    A = torch.diag(lam)
    for _ in range(reflections):
        v = torch.randn(N, dtype=torch.float64, device=device, generator=g)
        v /= v.norm()
        w = A @ v
        A += 4.0 * (v @ w) * torch.outer(v, v)
        A -= 2.0 * torch.outer(v, w)
        A -= 2.0 * torch.outer(w, v)
    return (A + A.T) / 2


def mimo_channels(batch, sizes=(4, 8, 16), rows_per_col=2, seed=1008, shuffle=True):
    """Channel matrices H (m = rows_per_col * N rows, N columns, iid CN(0,1)),
    the orders in equal shares, shuffled with the seed: the inputs of the
    MMSE filters W = (H^* H + s2 I)^{-1} H^*.  Returns (H flat complex128,
    n int32, m int32, hoff int64, woff int64): H_b row-major m x n at
    hoff[b], W_b row-major n x m at woff[b] (both packed back to back)."""
    rng = np.random.default_rng(seed)
    k = len(sizes)
    counts = [batch // k + (1 if i < batch % k else 0) for i in range(k)]
    n = np.concatenate([np.full(c, s, dtype=np.int32) for s, c in zip(sizes, counts)])
    if shuffle:
        n = n[rng.permutation(batch)]
    m = (rows_per_col * n).astype(np.int32)
    per = m.astype(np.int64) * n
    off = np.zeros(batch, dtype=np.int64)
    if batch > 1:
        off[1:] = np.cumsum(per)[:-1]
    total = int(per.sum())
    H = (rng.standard_normal(total) + 1j * rng.standard_normal(total)) * np.sqrt(0.5)
    return H, n, m, off, off.copy()
