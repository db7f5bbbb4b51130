"""FP64 pivots (Eq. 3) on inputs whose pivot cancels in FP32, and the
per-matrix automatic FP64-pivot pass (CHOL_FLAG_PIVOT64_AUTO), against the
oracle.

The inputs are A = D [[I, c], [c^*, d]] D with c exact in FP32 and the last
pivot's argument d - |c|^2 about 16 FP32 ulps of d (workloads.bordered_cancellation).
Every entry of R above the last pivot is then exact in FP32, so the error
of X comes from Eq. 3 alone: formed in FP32 the last pivot loses most of its
digits (the relative error of X is about that of the pivot, a few percent);
formed in FP64 from the exact products of the FP32 values it keeps them, and
X = [[I + c c^*/s, -c/s], [-c^*/s, 1/s]] (scaled) is then within a few FP32
rounding errors of the oracle: one rounding each for r_NN and 1/r_NN, then
a product or two per entry.  The bound checked is 32 u32.
"""
import numpy as np
import pytest

from paper_1111_4144_gb300 import workloads as wl

from gpu_helpers import U32, oracle_inv, run_inv, tol32, kappas, upper_errors

pytestmark = pytest.mark.gpu

BOUND64 = 32 * U32


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1111_4144_gb300 import _lib
    _lib.load()


def _redo_count():
    import ctypes
    from paper_1111_4144_gb300 import _lib as L
    c = ctypes.c_int64(0)
    L.check(L.chol_pivot64_redo_count(None, ctypes.byref(c)), "chol_pivot64_redo_count")
    return int(c.value)


def _errors_or_inf(b, X, Xo, info):
    e = upper_errors(b, X, Xo)
    e[(info != 0) | ~np.isfinite(e)] = np.inf
    return e


@pytest.mark.parametrize("tag", ["f32", "c64"])
@pytest.mark.parametrize("N", [6, 16, 24, 48])
def test_pivot64_recovers_cancelled_pivot(orc, tag, N):
    from paper_1111_4144_gb300 import _lib as L
    b = wl.bordered_cancellation(64, N, ratio=16.0, seed=300 + N, layout=1, complex_=(tag == "c64"))
    Ro, Xo, info_o, A_wide = oracle_inv(orc, b, tag)
    assert np.all(info_o == 0)
    X64, info64, R64 = run_inv(b, tag, mixed=False, want_R=True, flags=L.CHOL_FLAG_PIVOT64)
    assert np.all(info64 == 0)
    e64 = upper_errors(b, X64, Xo)
    assert np.all(e64 <= BOUND64), f"FP64 pivots: worst {e64.max():.3g} > {BOUND64:.3g}"
    assert np.all(upper_errors(b, R64, Ro) <= BOUND64)
    # the stated FP32 tolerance is met too (it is loose here: kappa is 1e7-1e9)
    assert np.all(e64 <= tol32(kappas(b, A_wide)))
    # FP32 pivots on the same inputs: breakdown, or errors orders of magnitude larger
    X32, info32, _ = run_inv(b, tag, mixed=False)
    e32 = _errors_or_inf(b, X32, Xo, info32)
    assert np.median(e32) > 100 * e64.max(), (np.median(e32), e64.max())


def _mixed_batch(N_hard, N_easy, tag, layout, seed):
    """Hard (cancelling) and easy (kappa = 100) matrices interleaved in one batch."""
    cplx = tag == "c64"
    hard = wl.bordered_cancellation(40, N_hard, ratio=16.0, seed=seed, layout=layout, complex_=cplx)
    easy = wl.fixed_kappa(40, N_easy, 100.0, seed=seed + 1, layout=layout)
    mats, n = [], []
    for k in range(40):
        for src in (hard, easy):
            N = int(src.n[k])
            per = N * (N + 1) // 2 if layout == 1 else N * N
            o = int(src.off[k])
            mats.append(src.A[o:o + per].astype(np.complex128 if cplx else np.float64))
            n.append(N)
    n = np.asarray(n, dtype=np.int32)
    off, _ = wl.layout_offsets(n, layout)
    return wl.Batch(np.concatenate(mats), n, off, layout), np.arange(0, 80, 2), np.arange(1, 80, 2)


@pytest.mark.parametrize("tag", ["f32", "c64"])
@pytest.mark.parametrize("Nh,Ne,layout", [(6, 6, 1), (16, 12, 1), (24, 30, 0), (48, 40, 0), (64, 64, 1)])
def test_pivot64_auto_redoes_only_cancelled(orc, tag, Nh, Ne, layout):
    from paper_1111_4144_gb300 import _lib as L
    b, hard, easy = _mixed_batch(Nh, Ne, tag, layout, seed=400 + Nh)
    mixed = Nh != Ne
    _, Xo, info_o, A_wide = oracle_inv(orc, b, tag)
    assert np.all(info_o == 0)
    Xp, infop, _ = run_inv(b, tag, mixed=mixed)
    _redo_count()  # clear the device counter
    Xa, infoa, _ = run_inv(b, tag, mixed=mixed, flags=L.CHOL_FLAG_PIVOT64_AUTO)
    assert _redo_count() == len(hard)
    assert np.all(infoa == 0)
    ea = upper_errors(b, Xa, Xo)
    # the easy matrices (kappa = 100 < 2^10) are never redone: bit for bit the plain result
    for k in easy:
        T = b.n[k] * (b.n[k] + 1) // 2 if layout == 1 else b.n[k] ** 2
        o = b.off[k]
        assert np.array_equal(Xa[o:o + T], Xp[o:o + T]), k
    assert np.all(ea[easy] <= tol32(kappas(b, A_wide))[easy])
    # the hard ones are redone with FP64 pivots and reach the FP64-pivot bound
    assert np.all(ea[hard] <= BOUND64), f"worst {ea[hard].max():.3g}"
    ep = _errors_or_inf(b, Xp, Xo, infop)
    assert np.median(ep[hard]) > 100 * ea[hard].max()


def test_pivot64_auto_matches_explicit_flag_on_the_warp_path(orc):
    """Orders 33-64 with CHOL_FLAG_PIVOT64 run the one-matrix-per-warp kernel,
    the same code as the redo pass: the two agree bit for bit."""
    from paper_1111_4144_gb300 import _lib as L
    b = wl.bordered_cancellation(50, 40, ratio=16.0, seed=505, layout=1)
    X64, info64, _ = run_inv(b, "f32", mixed=False, flags=L.CHOL_FLAG_PIVOT64)
    _redo_count()
    Xa, infoa, _ = run_inv(b, "f32", mixed=False, flags=L.CHOL_FLAG_PIVOT64_AUTO)
    assert _redo_count() == 50
    assert np.all(infoa == 0) and np.all(info64 == 0)
    assert np.array_equal(Xa, X64)


def test_pivot64_auto_non_pd_reports_info(orc):
    """A matrix that is not positive definite fails in the redo pass too:
    info is the failing row, the outputs are NaN."""
    from paper_1111_4144_gb300 import _lib as L
    b = wl.fixed_kappa(20, 20, 10.0, seed=9, layout=1)
    A = b.A.copy()
    k = 7
    o = int(b.off[k])
    # a_33 -> -a_33 (1-based row 3)
    pos = o + 2 * 20 - 1
    A[pos] = -abs(A[pos])
    b = wl.Batch(A, b.n, b.off, b.layout)
    _redo_count()
    X, info, _ = run_inv(b, "f32", mixed=False, flags=L.CHOL_FLAG_PIVOT64_AUTO)
    assert _redo_count() == 1
    _, _, info_o, _ = oracle_inv(orc, b, "f32")
    assert np.array_equal(info, info_o) and info[k] > 0
    T = 20 * 21 // 2
    assert np.all(np.isnan(X[o:o + T]))
