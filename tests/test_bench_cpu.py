"""The benchmark's host-side arithmetic on CPU: algorithmic bytes and flops
of the MIMO workload, the CUDA-core peak, the committed traffic record, the
error-over-tolerance ratio and the condition numbers it is scaled by."""
import hashlib
import json
import os

import numpy as np
import pytest

import bench
from paper_1111_4144_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _mimo_orders():
    # 1,048,576 matrices of orders 4, 8, 16 in equal shares (the first order takes the remainder)
    return np.concatenate([np.full(349526, 4), np.full(349525, 8), np.full(349525, 16)]).astype(np.int32)


def test_algorithmic_bytes_of_the_mimo_batch():
    # A's packed upper triangle read and X's written, 8 bytes per complex64 entry:
    # 160, 576 and 2176 bytes per matrix of order 4, 8, 16
    n = _mimo_orders()
    assert bench.alg_bytes(np.array([4]), 8) == 160
    assert bench.alg_bytes(np.array([8]), 8) == 576
    assert bench.alg_bytes(np.array([16]), 8) == 2176
    assert bench.alg_bytes(n, 8) == 349526 * 160 + 349525 * (576 + 2176) == 1_017_816_960


def test_algorithmic_flops_follow_table1_count():
    # (N^3 - N) / 2 multiply-adds per inverse (Table 1's n^3/2), 8 real flops per complex one
    assert bench.alg_flops(np.array([4]), cplx=True) == 8 * 30
    assert bench.alg_flops(np.array([16]), cplx=True) == 8 * 2040
    assert bench.alg_flops(np.array([64]), cplx=False) == 64 ** 3 - 64
    assert bench.alg_flops(_mimo_orders(), cplx=True) == 6_492_776_640
    assert bench.alg_flops(np.zeros(0, dtype=np.int32), cplx=False) == 0


def test_fp32_cuda_core_peak():
    # 152 SMs x 128 FP32 lanes x one FMA (2 flops) per clock at 2070 MHz
    assert bench.fp32_fma_peak_tflops(152) == pytest.approx(80.54784)
    assert bench.fp32_fma_peak_tflops(152, sm_mhz=1035.0) == pytest.approx(80.54784 / 2)


def test_measured_traffic_only_for_the_captured_sources():
    path = os.path.join(ROOT, "profiles", "k_group_c64_N16_traffic.json")
    rec = json.load(open(path))
    same = all(hashlib.sha256(open(os.path.join(ROOT, rel), "rb").read()).hexdigest() == h
               for rel, h in rec["source_sha256"].items())
    got = bench.measured_traffic(16, 349525)
    if same:
        assert got == pytest.approx(rec["dram_bytes_per_matrix"] * 349525)
        assert rec["dram_bytes_read"] + rec["dram_bytes_write"] == pytest.approx(
            rec["dram_bytes_per_matrix"] * rec["matrices"], rel=1e-6)
    else:
        assert got is None
    assert bench.measured_traffic(8, 349525) is None  # no capture of the order-8 kernel


def test_error_over_tolerance_ratio():
    b = wl.mimo_covariance(6, sizes=(2, 3), seed=5, layout=wl.LAYOUT_PACKED)
    Xo = b.A.astype(np.complex128) + 0.25
    Xg = Xo * (1 + 3e-8)  # relative Frobenius error 3e-8 in every matrix
    kap = np.array([1.0, 10.0, 1e3, 1e4, 2.0, 5e2])
    r, worst, med = bench.upper_err_ratio(b, Xg, Xo, kap, fp64=False)
    # FP32 tolerance max(1e-7 kappa, 2.4e-7): the smallest tolerance (2.4e-7) gives the largest ratio
    assert worst == pytest.approx(3e-8, rel=1e-6) and med == pytest.approx(3e-8, rel=1e-6)
    assert r == pytest.approx(3e-8 / 2.4e-7, rel=1e-6)
    r64, _, _ = bench.upper_err_ratio(b, Xg, Xo, kap, fp64=True)
    assert r64 == pytest.approx(3e-8 / 1e-11, rel=1e-6)


def test_condition_numbers_of_packed_matrices():
    # diag(1, 100) and a Hermitian 2 x 2 with eigenvalues 1 and 3
    A = np.array([1.0, 0.0, 100.0, 2.0, 1j, 2.0], dtype=np.complex128)
    b = wl.Batch(A, np.array([2, 2], dtype=np.int32), np.array([0, 3], dtype=np.int64), wl.LAYOUT_PACKED)
    assert bench.kappa_of(b, A) == pytest.approx([100.0, 3.0])


def test_single_thread_oracle_timing_on_a_prefix(orc):
    """The one-thread oracle figure runs on the first matrices of the batch
    (a contiguous prefix of the packed buffer) and inverts them correctly."""
    b = wl.mimo_covariance(300, sizes=(4, 8, 16), seed=7, layout=wl.LAYOUT_PACKED)
    A = b.A.astype(np.complex64).astype(np.complex128)
    v, count, reps = bench.oracle_time_single(b, A, 100, min_wall=0.0)
    assert count == 100 and reps >= 1 and v > 0
    v, count, _ = bench.oracle_time_single(b, A, 10 ** 6, min_wall=0.0)
    assert count == 300
    last = int(b.n[99])
    end = int(b.off[99]) + last * (last + 1) // 2
    _, X1, info1 = orc.inv_batch(A[:end], b.n[:100], b.off[:100], 1, True, nthreads=1)
    _, Xa, infoa = orc.inv_batch(A, b.n, b.off, 1, True)
    assert np.all(info1 == 0) and np.array_equal(X1, Xa[:end])
