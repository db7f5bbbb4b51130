"""GPU parity: the batched CUDA path (through the C ABI) against the CPU oracle.

Inputs come from the seeded generators; both sides see the same matrices
rounded to the working precision.  Per-matrix relative Frobenius error over
the upper triangle must stay within: 1e-11 (FP64 / complex128) and
max(1e-7 * kappa, 2.4e-7) (FP32 / complex64, kappa the 2-norm condition
number of the rounded matrix).
"""
import numpy as np
import pytest

from paper_1111_4144_gb300 import workloads as wl

from gpu_helpers import TOL64, cast_batch, check_errors, kappas, oracle_inv, run_inv, tol32, upper_errors

pytestmark = pytest.mark.gpu

TAGS = ["f32", "f64", "c64", "c128"]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1111_4144_gb300 import _lib
    _lib.load()


def make_batch(tag, N, batch, layout, seed):
    if tag in ("c64", "c128"):
        return wl.mimo_covariance(batch, sizes=(N,), seed=seed, layout=layout, shuffle=False)
    return wl.qr_spectrum(batch, lambda rng, b: np.full(b, N),
                          lambda rng, m, NN: 10.0 ** rng.uniform(0.0, 3.0, size=(m, NN)), seed, layout)


@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 8, 11, 15, 16, 17, 24, 32, 33, 48, 63, 64])
@pytest.mark.parametrize("tag", TAGS)
def test_uniform_parity(orc, tag, N, layout):
    batch = 300 if N <= 32 else 90
    b = make_batch(tag, N, batch, layout, seed=1000 + N)
    X, info, R = run_inv(b, tag, mixed=False, want_R=True)
    Ro, Xo, info_o, A_wide = oracle_inv(orc, b, tag)
    assert np.all(info_o == 0) and np.array_equal(info, info_o)
    check_errors(tag, b, A_wide, upper_errors(b, X, Xo), "X")
    check_errors(tag, b, A_wide, upper_errors(b, R, Ro), "R")
    if layout == 0:
        # dense R: strictly lower part written as zero
        for k in range(0, batch, 37):
            M = R[b.off[k]:b.off[k] + N * N].reshape(N, N)
            assert np.all(np.tril(M, -1) == 0)


@pytest.mark.parametrize("tag,kind", [("c64", "mimo"), ("c128", "mimo"), ("f32", "uneven"), ("f64", "uneven"),
                                      ("c64", "uneven_c")])
def test_mixed_sizes_parity(orc, tag, kind):
    if kind == "mimo":
        b = wl.mimo_covariance(3001, sizes=(4, 8, 16), seed=1001, layout=1)
    elif kind == "uneven":
        b = wl.uneven_loguniform(700, nmin=2, nmax=64, seed=1002, layout=0)
    else:
        b = wl.mimo_covariance(900, sizes=tuple(range(1, 41)), seed=77, layout=0)
    X, info, _ = run_inv(b, tag, mixed=True)
    Ro, Xo, info_o, A_wide = oracle_inv(orc, b, tag)
    assert np.all(info_o == 0) and np.array_equal(info, info_o)
    check_errors(tag, b, A_wide, upper_errors(b, X, Xo), "X")


@pytest.mark.parametrize("tag", ["f32", "c128"])
def test_fill_lower(orc, tag):
    b = make_batch(tag if tag != "f32" else "f32", 12, 50, 0, seed=5)
    X, _, _ = run_inv(b, tag, mixed=False, fill_lower=True)
    for k in range(b.batch):
        M = X[b.off[k]:b.off[k] + 144].reshape(12, 12)
        assert np.array_equal(np.tril(M, -1), np.conj(np.triu(M, 1)).T)


@pytest.mark.parametrize("tag", TAGS)
def test_non_pd_info_and_nan_fill(orc, tag):
    N = 6
    b = make_batch(tag, N, 40, 0, seed=9)
    A = b.A.copy()
    bad = {3: 1, 17: 4, 39: 6}
    for k, row in bad.items():
        o = b.off[k]
        M = A[o:o + N * N].reshape(N, N)
        M[row - 1, row - 1] = -abs(M[row - 1, row - 1]) * 50.0  # destroys positive definiteness at that row
    b2 = wl.Batch(A, b.n, b.off, 0)
    X, info, _ = run_inv(b2, tag, mixed=False)
    _, _, info_o, _ = oracle_inv(orc, b2, tag)
    assert np.array_equal(info, info_o)
    for k, row in bad.items():
        assert info[k] == row
        M = X[b.off[k]:b.off[k] + N * N].reshape(N, N)
        assert np.all(np.isnan(M[np.triu_indices(N)].real))
    good = [k for k in range(b.batch) if k not in bad]
    assert np.all(info[good] == 0)


def test_zero_and_invalid_sizes(orc):
    import torch
    from paper_1111_4144_gb300 import _lib as L, api
    b = wl.mimo_covariance(64, sizes=(5, 7), seed=3, layout=1)
    n = b.n.copy()
    n[10] = 0
    A_np = b.A.astype(np.complex64)
    dev = torch.device("cuda", 0)
    A = torch.from_numpy(A_np).to(dev)
    X0 = torch.full_like(A, 7.0)
    api.inv(A, torch.from_numpy(n).to(dev), torch.from_numpy(b.off).to(dev), 8, layout=1, X=X0)
    torch.cuda.synchronize()
    assert api.last_device_error() == L.CHOL_OK
    n2 = n.copy()
    n2[20] = 9  # larger than max_n = 8
    X1 = torch.full_like(A, 7.0)
    _, info = api.inv(A, torch.from_numpy(n2).to(dev), torch.from_numpy(b.off).to(dev), 8, layout=1, X=X1)
    info = info.cpu().numpy()
    assert info[20] == -1 and info[10] == 0
    assert api.last_device_error() == L.CHOL_ERR_ARG
    assert api.last_device_error() == L.CHOL_OK  # the error word was cleared by the read
    X1 = X1.cpu().numpy()
    o = b.off[10]
    assert np.all(X1[o:o + 15] == 7.0)  # the empty matrix's slots were not written


@pytest.mark.parametrize("tag,kind", [("c64", "mimo"), ("f32", "uneven")])
def test_plan_replay_matches_eager(orc, tag, kind):
    if kind == "mimo":
        b = wl.mimo_covariance(5000, sizes=(4, 8, 16), seed=11, layout=1)
    else:
        b = wl.uneven_loguniform(400, seed=12, layout=0)
    Xe, ie, _ = run_inv(b, tag, mixed=True)
    Xp, ip, _ = run_inv(b, tag, mixed=True, plan=True)
    assert np.array_equal(ie, ip)
    assert np.array_equal(Xe.view(np.uint8), Xp.view(np.uint8))


@pytest.mark.parametrize("tag", ["f64", "c64"])
@pytest.mark.parametrize("N", [6, 20])
def test_in_place_x_equals_a(orc, tag, N):
    import torch
    from paper_1111_4144_gb300 import api
    b = make_batch(tag, N, 64, 1, seed=21)
    A_np, _ = cast_batch(b, tag)
    A = torch.from_numpy(A_np).cuda()
    api.inv(A, max_n=N, layout=1, X=A)
    torch.cuda.synchronize()
    _, Xo, _, A_wide = oracle_inv(orc, b, tag)
    check_errors(tag, b, A_wide, upper_errors(b, A.cpu().numpy(), Xo), "X (in place)")


@pytest.mark.parametrize("tag", TAGS)
@pytest.mark.parametrize("N", [7, 40])
def test_factor_only(orc, tag, N):
    import torch
    from paper_1111_4144_gb300 import api
    b = make_batch(tag, N, 70, 0, seed=31)
    A_np, _ = cast_batch(b, tag)
    A = torch.from_numpy(A_np).cuda()
    R, info = api.factor(A, max_n=N, layout=0)
    torch.cuda.synchronize()
    Ro, _, info_o, A_wide = oracle_inv(orc, b, tag)
    assert np.array_equal(info.cpu().numpy(), info_o)
    R = R.cpu().numpy()
    check_errors(tag, b, A_wide, upper_errors(b, R, Ro), "R")
    for k in range(0, b.batch, 9):
        M = R[b.off[k]:b.off[k] + N * N].reshape(N, N)
        assert np.all(np.tril(M, -1) == 0)


def test_empty_batch():
    from paper_1111_4144_gb300 import _lib as L
    o = L.opts()
    assert L.chol_inv_batched(L.CHOL_F32, 0, None, None, 4, None, None, None, None, o, None, 0, None) == L.CHOL_OK


def test_plan_fixed_orders():
    """CHOL_FLAG_PLAN_ORDERS: kernels only for the orders present at creation;
    bit-identical to the eager call; a matrix whose order appears only later
    is rejected (info -1, device error word) and the others are unaffected."""
    import torch
    from paper_1111_4144_gb300 import _lib as L, api
    b = wl.mimo_covariance(6000, sizes=(4, 8, 16), seed=14, layout=1)
    Xe, ie, _ = run_inv(b, "c64", mixed=True)
    A = torch.from_numpy(b.A.astype(np.complex64)).cuda()
    n = torch.from_numpy(b.n).cuda()
    off = torch.from_numpy(b.off).cuda()
    X = torch.zeros_like(A)
    api.last_device_error()  # clear
    p = api.Plan(A, X, n, off, 16, layout=1, fixed_orders=True, timing=True)
    p.launch()
    torch.cuda.synchronize()
    assert np.array_equal(p.info.cpu().numpy(), ie)
    assert np.array_equal(X.cpu().numpy().view(np.uint8), Xe.view(np.uint8))
    with pytest.raises(L.CholError):
        p.kernel_ms(5)  # no kernel recorded for an absent order
    # matrix 0 (order n0) becomes an order-3 matrix in the same storage
    k = 0
    n0 = int(b.n[k])
    n[k] = 3
    X.zero_()
    p.launch()
    torch.cuda.synchronize()
    info = p.info.cpu().numpy()
    assert info[k] == -1 and np.all(info[1:] == ie[1:])
    assert api.last_device_error() == L.CHOL_ERR_ARG
    Xg = X.cpu().numpy()
    for j in range(1, b.batch, 97):
        o, T = int(b.off[j]), int(b.n[j]) * (int(b.n[j]) + 1) // 2
        assert np.array_equal(Xg[o:o + T].view(np.uint8), Xe[o:o + T].view(np.uint8))
    assert n0 in (4, 8, 16)
    p.close()


def test_forked_classes_match_sequential(orc):
    """Many orders (2..64): the class kernels run side by side on forked
    streams (eager call, and parallel branches of a plan); a timing plan runs
    them one after another.  All three give bit-identical X and info, and X
    matches the oracle."""
    import torch
    from paper_1111_4144_gb300 import api
    b = wl.uneven_loguniform(3000, nmin=2, nmax=64, seed=21, layout=0)
    A_np, _ = cast_batch(b, "f32")
    A = torch.from_numpy(A_np).cuda()
    n = torch.from_numpy(b.n).cuda()
    off = torch.from_numpy(b.off).cuda()
    outs = []
    for timing in (False, True):
        X = torch.full_like(A, float("nan"))
        p = api.Plan(A, X, n, off, 64, fixed_orders=True, timing=timing)
        p.launch()
        p.launch()
        torch.cuda.synchronize()
        outs.append((X.cpu().numpy(), p.info.cpu().numpy()))
        p.close()
    Xe, ie, _ = run_inv(b, "f32", mixed=True)
    for Xg, ig in outs:
        assert np.array_equal(ig, ie)
        for k in range(b.batch):
            o, N = int(b.off[k]), int(b.n[k])
            got = np.triu(Xg[o:o + N * N].reshape(N, N))
            want = np.triu(Xe[o:o + N * N].reshape(N, N))
            assert np.array_equal(got.view(np.uint32), want.view(np.uint32)), k
    Ro, Xo, info_o, A_wide = oracle_inv(orc, b, "f32")
    check_errors("f32", b, A_wide, upper_errors(b, Xe, Xo), "X")


def test_plan_kernel_timing():
    import torch
    from paper_1111_4144_gb300 import api
    b = wl.mimo_covariance(20000, sizes=(4, 8, 16), seed=13, layout=1)
    A = torch.from_numpy(b.A.astype(np.complex64)).cuda()
    n = torch.from_numpy(b.n).cuda()
    off = torch.from_numpy(b.off).cuda()
    X = torch.zeros_like(A)
    p = api.Plan(A, X, n, off, 16, layout=1, timing=True)
    p.launch()
    torch.cuda.synchronize()
    for N in (4, 8, 16):
        assert p.kernel_ms(N) > 0.0
    p.close()


@pytest.mark.parametrize("tag", ["c64", "f32", "c128"])
def test_every_kernel_variant_matches_oracle(orc, tag):
    """Each compiled variant of an order (lane / group G / group 2G) gives results
    within tolerance; the tuning table is restored afterwards."""
    from paper_1111_4144_gb300 import _lib as L
    dt = {"f32": L.CHOL_F32, "c64": L.CHOL_C64, "c128": L.CHOL_C128}[tag]
    try:
        for N in (8, 9, 12, 16, 20, 32):
            nv = L.chol_tune_variants(dt, N)
            assert nv >= 1
            b = make_batch(tag, N, 150, 1, seed=300 + N)
            Ro, Xo, info_o, A_wide = oracle_inv(orc, b, tag)
            for v in range(nv):
                assert L.chol_tune_set(dt, N, v) == L.CHOL_OK
                X, info, _ = run_inv(b, tag, mixed=False)
                assert np.array_equal(info, info_o)
                check_errors(tag, b, A_wide, upper_errors(b, X, Xo), f"X (N={N}, variant {v})")
            assert L.chol_tune_set(dt, N, nv) == L.CHOL_ERR_ARG
    finally:
        for N in range(1, 65):
            L.chol_tune_set(dt, N, 0)


def test_autotune_and_cache(tmp_path):
    from paper_1111_4144_gb300 import _lib as L, api
    import torch
    path = str(tmp_path / "tune.txt")
    chosen = api.autotune(torch.complex64, 16, layout=1, batch=4096, cache_path=path)
    assert set(chosen) == {n for n in range(1, 17) if L.chol_tune_variants(L.CHOL_C64, n) > 1}
    text = open(path).read()
    assert text.startswith("device ")
    for n in chosen:
        L.chol_tune_set(L.CHOL_C64, n, 0)
    assert L.chol_tune_load(path.encode()) == L.CHOL_OK
    assert {n: L.chol_tune_get(L.CHOL_C64, n) for n in chosen} == chosen
    for n in chosen:
        L.chol_tune_set(L.CHOL_C64, n, 0)


@pytest.mark.parametrize("layout", [0, 1])
def test_wide_kernel_every_order(orc, layout):
    """FP32 orders 33..64: the register-resident one-warp-per-matrix kernel
    (variant 0) and the shared-memory warp kernel (variant 1), each against
    the oracle at every order, with a ragged last chunk (CTAs take four
    matrices), R written and, in the dense layout, the lower half of X
    filled."""
    from paper_1111_4144_gb300 import _lib as L
    try:
        for N in range(33, 65):
            assert L.chol_tune_variants(L.CHOL_F32, N) == 2
            b = make_batch("f32", N, 37 + N % 4, layout, seed=600 + N)
            Ro, Xo, info_o, A_wide = oracle_inv(orc, b, "f32", fill_lower=(layout == 0))
            for v in (0, 1):
                assert L.chol_tune_set(L.CHOL_F32, N, v) == L.CHOL_OK
                X, info, R = run_inv(b, "f32", mixed=False, want_R=True, fill_lower=(layout == 0))
                assert np.array_equal(info, info_o)
                check_errors("f32", b, A_wide, upper_errors(b, X, Xo), f"X (N={N}, variant {v})")
                check_errors("f32", b, A_wide, upper_errors(b, R, Ro), f"R (N={N}, variant {v})")
                if layout == 0:
                    for k in (0, b.batch - 1):
                        M = X[b.off[k]:b.off[k] + N * N].reshape(N, N)
                        assert np.array_equal(M, M.T)
    finally:
        for N in range(33, 65):
            L.chol_tune_set(L.CHOL_F32, N, 0)


@pytest.mark.parametrize("N", [33, 47, 64])
def test_wide_kernel_in_place_and_factor_only(orc, N):
    import torch
    from paper_1111_4144_gb300 import api
    b = make_batch("f32", N, 45, 1, seed=700 + N)
    A_np, _ = cast_batch(b, "f32")
    Ro, Xo, info_o, A_wide = oracle_inv(orc, b, "f32")
    A = torch.from_numpy(A_np).cuda()
    R, info = api.factor(A, max_n=N, layout=1)
    torch.cuda.synchronize()
    assert np.array_equal(info.cpu().numpy(), info_o)
    check_errors("f32", b, A_wide, upper_errors(b, R.cpu().numpy(), Ro), "R (factor only)")
    api.inv(A, max_n=N, layout=1, X=A)  # X == A
    torch.cuda.synchronize()
    check_errors("f32", b, A_wide, upper_errors(b, A.cpu().numpy(), Xo), "X (in place)")


@pytest.mark.parametrize("method", ["es", "tmo"])
@pytest.mark.parametrize("tag", TAGS)
def test_comparison_methods_match_oracle(orc, tag, method):
    """The paper's existing methods on the GPU (Sec. III.A Equation Solving,
    Sec. III.B Triangular Matrix Operations), one matrix per warp, mixed
    orders 1..64: X within the tolerance of the oracle's own ES / TMO (and so
    of the proposed method's X, which both pins tie to the same inverse)."""
    from paper_1111_4144_gb300 import _lib as L
    flag = L.CHOL_FLAG_METHOD_ES if method == "es" else L.CHOL_FLAG_METHOD_TMO
    b = wl.uneven_loguniform(200, nmin=1, nmax=64, seed=2200 if method == "es" else 2201, layout=1)
    if tag in ("c64", "c128"):
        mc = wl.mimo_covariance(200, sizes=(3, 17, 40, 64), seed=2202, layout=1)
        b = mc
    X, info, _ = run_inv(b, tag, mixed=True, flags=flag)
    _, Xo, info_o, A_wide = oracle_inv(orc, b, tag)
    assert np.array_equal(info, info_o) and np.all(info == 0)
    # the oracle's ES / TMO on every matrix
    bb = wl.Batch(A_wide, b.n, b.off, b.layout)
    ref = np.zeros_like(Xo)
    for k in range(b.batch):
        N = int(b.n[k])
        M = bb.matrix(k)
        M = np.triu(M) + np.conj(np.triu(M, 1)).T
        Rk, inf = orc.chol(M)
        Xk = orc.es(Rk) if method == "es" else orc.tmo(Rk)
        iu = np.triu_indices(N)
        ref[b.off[k]:b.off[k] + N * (N + 1) // 2] = Xk[iu]
    check_errors(tag, b, A_wide, upper_errors(b, X, ref), f"X ({method})")
    check_errors(tag, b, A_wide, upper_errors(b, X, Xo), f"X ({method}) vs proposed")


@pytest.mark.parametrize("tag", ["f64", "c128"])
def test_equation_solving_equals_proposed_bits(tag):
    """ES's forward solve gives b_i = 0 (i < j) and b_j = 1/r_jj, the s_ij of
    Eq. 24, after which its back substitution takes the proposed method's
    steps: on the same one-matrix-per-warp kernel (FP64 orders above 32 run
    it by default) the two agree bit for bit, as they do in the oracle."""
    from paper_1111_4144_gb300 import _lib as L
    b = make_batch(tag, 41, 70, 1, seed=2203)
    Xp, ip, _ = run_inv(b, tag, mixed=False)
    Xe, ie, _ = run_inv(b, tag, mixed=False, flags=L.CHOL_FLAG_METHOD_ES)
    assert np.all(ip == 0) and np.array_equal(ip, ie)
    assert np.array_equal(Xp, Xe)


@pytest.mark.parametrize("tag,kind", [("f32", "uneven"), ("c64", "mimo"), ("f64", "uneven"), ("f32", "uniform")])
def test_single_launch_matches_oracle(orc, tag, kind):
    """CHOL_FLAG_SINGLE_LAUNCH: the whole batch in one persistent launch,
    largest orders first, each matrix at its own order: eager and plan
    replay against the oracle."""
    from paper_1111_4144_gb300 import _lib as L
    if kind == "uneven":
        b = wl.uneven_loguniform(700, nmin=1, nmax=64, seed=2300, layout=0)
    elif kind == "mimo":
        b = wl.mimo_covariance(900, sizes=(4, 8, 16), seed=2301, layout=1)
    else:
        b = make_batch(tag, 37, 101, 1, seed=2302)
    mixed = kind != "uniform"
    _, Xo, info_o, A_wide = oracle_inv(orc, b, tag)
    for plan in (False, True):
        X, info, _ = run_inv(b, tag, mixed=mixed, plan=plan, flags=L.CHOL_FLAG_SINGLE_LAUNCH)
        assert np.array_equal(info, info_o)
        check_errors(tag, b, A_wide, upper_errors(b, X, Xo), f"X (single launch, plan={plan})")


def _class_kernel_launches(fn):
    """Names of the size-class kernels (k_lane / k_group / k_wide / k_warp)
    that fn() launched, from the CUDA activity of torch's profiler; None if
    the profiler records no CUDA activity here."""
    import torch
    from torch.profiler import ProfilerActivity, profile
    torch.cuda.synchronize()
    try:
        with profile(activities=[ProfilerActivity.CUDA]) as prof:
            fn()
            torch.cuda.synchronize()
        names = [e.name for e in prof.events() if e.device_type == torch.autograd.DeviceType.CUDA]
    except RuntimeError:
        return None
    if not names:
        return None
    return [s for s in names if any(k in s for k in ("k_lane", "k_group", "k_wide", "k_warp"))]


def test_order_set_launches_only_stated_orders(orc):
    """chol_opts_t.orders: an eager call on a batch of orders {4, 8, 16}
    launches those three size-class kernels only, with results bit-identical
    to the call without the set; a matrix of an order outside the set gets
    info = -1 and the device error word CHOL_ERR_ARG."""
    import torch
    from paper_1111_4144_gb300 import _lib as L, api
    b = wl.mimo_covariance(3000, sizes=(4, 8, 16), seed=2401, layout=1)
    dev = torch.device("cuda", 0)
    A = torch.from_numpy(b.A.astype(np.complex64)).to(dev)
    n = torch.from_numpy(b.n).to(dev)
    off = torch.from_numpy(b.off).to(dev)
    api.last_device_error()  # clear
    X0, i0 = api.inv(A, n, off, 16, layout=1)
    X1, i1 = api.inv(A, n, off, 16, layout=1, orders=(4, 8, 16))
    torch.cuda.synchronize()
    assert torch.equal(i0, i1) and int(i1.abs().sum()) == 0
    assert torch.equal(X0.view(torch.float32), X1.view(torch.float32))
    assert api.last_device_error() == L.CHOL_OK
    # the same through a plan (the set restricts every replay)
    Xp = torch.zeros_like(A)
    p = api.Plan(A, Xp, n, off, 16, layout=1, orders=(4, 8, 16))
    p.launch()
    torch.cuda.synchronize()
    assert torch.equal(X0.view(torch.float32), Xp.view(torch.float32))
    p.close()
    # launches: three class kernels with the set, one per order 1..16 without
    stated = _class_kernel_launches(lambda: api.inv(A, n, off, 16, layout=1, orders=(4, 8, 16)))
    every = _class_kernel_launches(lambda: api.inv(A, n, off, 16, layout=1))
    if stated is not None:
        assert len(stated) == 3, stated
        assert len(every) == 16, every
    # order 16 left out of the set: its matrices are rejected, the rest unchanged
    X2, i2 = api.inv(A, n, off, 16, layout=1, orders=(4, 8))
    torch.cuda.synchronize()
    i2 = i2.cpu().numpy()
    assert np.all(i2[b.n == 16] == -1) and np.all(i2[b.n != 16] == 0)
    assert api.last_device_error() == L.CHOL_ERR_ARG
    Xa, Xb = X0.cpu().numpy(), X2.cpu().numpy()
    for k in np.flatnonzero(b.n != 16)[:200]:
        o, T = int(b.off[k]), int(b.n[k]) * (int(b.n[k]) + 1) // 2
        assert np.array_equal(Xa[o:o + T], Xb[o:o + T])
