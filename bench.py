#!/usr/bin/env python
"""Throughput benchmark: batched Cholesky + direct inverse of 1,048,576 complex
MIMO covariance matrices (N in {4, 8, 16}, one third each, shuffled;
A = H^H H + 0.1 I with H a 2N x N matrix of iid CN(0,1) entries), complex64
inputs and FP32 arithmetic, upper triangles packed, one CUDA-graph replay per
step.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU FP64 oracle (the plain C implementation the
tests check against) on this machine's host cores.  Under torchrun each rank
inverts its own batch (weak scaling; no data-path collective).

After the timed legs, rank 0 adds a `configs` object that times the other
batched workloads (4,096 FP64 order-8 matrices; 262,144 FP32 matrices of
orders 2..64; forward + adjoint of 65,536 FP32 order-32 matrices), each with
an oracle sample as its CPU baseline and accuracy check; --no-extra skips it.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BATCH = 1 << 20
SIZES = (4, 8, 16)
SIGMA2 = 0.1
SEED = 1001
METRIC = "inverses/s"
WORKLOAD = "mimo_covariance_c64_N4-8-16_x1048576_packed"
FALLBACK_HBM_GBS = 6800.0
FALLBACK_BF16_TFLOPS = 1900.0
FALLBACK_BF16_TFLOPS_SUSTAINED = 1700.0
TF32_OVER_BF16 = 1.1 / 2.25  # nominal dense TF32 : BF16 tensor rates


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--quick", action="store_true",
                    help="time the device step only (no accuracy check, FP64 form, e2e or CPU baseline); "
                         "for profiler runs")
    ap.add_argument("--batch", type=int, default=BATCH, help="matrices per GPU (profiling cases)")
    ap.add_argument("--sizes", default=",".join(map(str, SIZES)), help="matrix orders, equal shares")
    ap.add_argument("--uniform", action="store_true",
                    help="profiling case: one order only (first of --sizes), no per-matrix sizes")
    ap.add_argument("--blocked", type=int, default=0,
                    help="time the blocked path instead: one FP32 matrix of this order, lambda log-spaced over "
                         "[1, 1e4], tensor-core products (prints one JSON line)")
    ap.add_argument("--blocked-prec", default="tf32", choices=["tf32", "fp32", "fp64"])
    ap.add_argument("--blocked-pivots", default="fp64", choices=["fp64", "fp32"],
                    help="pivots of the FP32 / TF32 blocked run: FP64 (the large workload's setting) or FP32")
    ap.add_argument("--blocked-refine", type=int, default=2,
                    help="refinement steps of the FP32 / TF32 blocked run (the large workload takes 2, with FP64 "
                         "pivots)")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the other workloads (FP64 order 8, uneven FP32, forward + adjoint, refinement, "
                         "large blocked)")
    ap.add_argument("--no-blocked", action="store_true", help="skip the large blocked workloads (N = 4096, 16384)")
    ap.add_argument("--profile-case", default="",
                    help="profiling case DTYPE:N:BATCH (e.g. f32:64:32768): a uniform packed batch of real SPD "
                         "(lambda log-uniform in [1, 1e3]) or complex MIMO matrices through the default kernel of "
                         "that order, --steps launches inside an NVTX range 'step'; prints the mean time")
    return ap.parse_args()


def tri(n):
    return n * (n + 1) // 2


def alg_bytes(n, elem_bytes):
    """Algorithmic bytes of one pass: the upper triangle of A read, that of X written."""
    t = (np.asarray(n, dtype=np.int64) * (np.asarray(n, dtype=np.int64) + 1)) // 2
    return int(2 * t.sum() * elem_bytes)


def alg_flops(n, cplx=True):
    """Algorithmic flops: (N^3 - N)/2 multiply-adds per matrix (Table 1's 1/2 n^3),
    a complex multiply-add counted as 8 real flops."""
    n = np.asarray(n, dtype=np.int64)
    macs = ((n ** 3 - n) // 2).sum()
    return int(macs * (8 if cplx else 2))


def fp32_fma_peak_tflops(sms, sm_mhz=2070.0):
    """FP32 CUDA-core peak: every SM's 128 FP32 lanes retire one fused
    multiply-add (2 flops) per clock, at the maximum SM clock."""
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p)), "measured"
        except Exception:
            pass
    return {"hbm_gbs": FALLBACK_HBM_GBS}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while the GPU is busy."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.index)], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [r for r in rows if r[2] > 0.5 * max(x[2] for x in rows)] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in loaded for i, v in enumerate(r[3]) if v.lower() == "active"})
        return {"sm_mhz": float(np.median([r[0] for r in loaded])), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(loaded), "power_w_max": max(r[2] for r in rows)}


def max_over_ranks(ms, world, device):
    """The job's step time: the slowest rank's (all-reduce MAX; a no-op on one rank)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, batch_per_rank, ms):
    """Whole-job throughput (weak scaling): every rank inverts its own batch."""
    return world * batch_per_rank / (ms / 1e3)


def make_workload(rank, batch=BATCH, sizes=SIZES):
    """Rank `rank`'s shard: its own seeded batch (no data moves between ranks)."""
    from paper_1111_4144_gb300 import workloads as wl
    return wl.mimo_covariance(batch, sizes=sizes, sigma2=SIGMA2, seed=SEED + rank, layout=wl.LAYOUT_PACKED)


def oracle_time(b, A_wide, min_wall=1.0):
    """Time the CPU oracle on this batch; returns (inverses/s, threads, reps, result)."""
    import oracle
    threads = os.cpu_count() or 1
    reps, t0 = 0, time.perf_counter()
    res = None
    while True:
        res = oracle.inv_batch(A_wide, b.n, b.off, 1, True, nthreads=threads)
        reps += 1
        el = time.perf_counter() - t0
        if el >= min_wall:
            break
    return reps * b.batch / el, threads, reps, res


def oracle_time_single(b, A_wide, count, min_wall=0.5):
    """The oracle on one thread over the batch's first `count` matrices (stored
    back to back from offset 0); returns (inverses/s, matrices, passes)."""
    import oracle
    count = min(count, b.batch)
    last = int(b.n[count - 1])
    end = int(b.off[count - 1]) + (last * (last + 1) // 2 if b.layout else last * last)
    A = np.ascontiguousarray(A_wide[:end])
    cplx = np.iscomplexobj(A_wide)
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle.inv_batch(A, b.n[:count], b.off[:count], b.layout, cplx, nthreads=1)
        reps += 1
        el = time.perf_counter() - t0
        if el >= min_wall:
            break
    return reps * count / el, count, reps


def upper_err_ratio(b, Xg, Xo, kappa, fp64):
    """max over matrices of (relative Frobenius error of the upper triangle) / tolerance."""
    n = b.n.astype(np.int64)
    t = n * (n + 1) // 2
    seg = np.repeat(np.arange(b.batch), t)
    d = np.abs(Xg.astype(np.complex128) - Xo) ** 2
    num = np.sqrt(np.bincount(seg, weights=d, minlength=b.batch))
    den = np.sqrt(np.bincount(seg, weights=np.abs(Xo) ** 2, minlength=b.batch))
    err = num / den
    tol = np.full(b.batch, 1e-11) if fp64 else np.maximum(1e-7 * kappa, 2.4e-7)
    return float(np.max(err / tol)), float(np.max(err)), float(np.median(err))


def kappa_of(b, A_wide):
    """2-norm condition numbers of the packed Hermitian matrices."""
    from paper_1111_4144_gb300 import workloads as wl
    kap = np.zeros(b.batch)
    for N in np.unique(b.n):
        idx = np.nonzero(b.n == N)[0]
        iu = np.triu_indices(N)
        M = np.zeros((len(idx), N, N), dtype=np.complex128)
        pos = b.off[idx][:, None] + np.arange(wl.tri(N))[None, :]
        M[:, iu[0], iu[1]] = A_wide[pos]
        M = M + np.conj(np.transpose(np.triu(M, 1), (0, 2, 1)))
        ev = np.linalg.eigvalsh(M)
        kap[idx] = ev[:, -1] / ev[:, 0]
    return kap


def run_reference(args, rank, world):
    if rank != 0:
        return
    sizes = tuple(int(x) for x in args.sizes.split(","))
    b = make_workload(0, args.batch, sizes)
    A_wide = b.A.astype(np.complex64).astype(np.complex128)
    t_start = time.perf_counter()
    per = []
    threads = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle_time(b, A_wide, min_wall=0.0)
    for _ in range(args.steps):
        v, threads, reps, _ = oracle_time(b, A_wide, min_wall=0.0)
        per.append(b.batch / v)
    ms = 1e3 * float(np.mean(per))
    value = b.batch / (ms / 1e3)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD if b.batch == BATCH and sizes == SIZES else
                       f"mimo_covariance_c64_N{'-'.join(map(str, sizes))}_x{b.batch}_packed",
                       "batch": b.batch, "sizes": list(sizes), "layout": "packed_upper"},
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": threads, "kind": "oracle",
                             "sample": f"full {b.batch}-matrix batch per step, FP64 oracle, {threads} threads"},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t_start}
    print(json.dumps(line), flush=True)


def measured_traffic(order, count):
    """DRAM bytes of one launch of the order-`order` complex64 kernel, from the
    committed ncu capture (per-matrix traffic x matrices), or None when no
    capture matches the current kernel sources."""
    import hashlib
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "profiles", "k_group_c64_N16_traffic.json")
    if order != 16 or not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f)
    root = os.path.dirname(path)
    for rel, digest in rec["source_sha256"].items():
        with open(os.path.join(root, "..", rel), "rb") as src:
            if hashlib.sha256(src.read()).hexdigest() != digest:
                return None
    return rec["dram_bytes_per_matrix"] * count


def host_link_ceiling(dev, A_h, X_h, A, X, reps=5):
    """The host link alone: pinned cudaMemcpyAsync of the step's input (host to
    device) and of its output (device to host), each direction alone and
    both at once on two streams, timed with CUDA events (the copies of the
    end-to-end step with no kernel).  Returns ms and GB/s."""
    import torch
    s1, s2 = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)

    def run(h2d, d2h):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s1)
        s2.wait_event(e0)
        for _ in range(reps):
            if h2d:
                with torch.cuda.stream(s1):
                    A.copy_(A_h, non_blocking=True)
            if d2h:
                with torch.cuda.stream(s2):
                    X_h.copy_(X, non_blocking=True)
        s1.wait_stream(s2)
        e1.record(s1)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    run(True, True)
    h, d, both = run(True, False), run(False, True), run(True, True)
    nb_in, nb_out = A_h.numel() * A_h.element_size(), X_h.numel() * X_h.element_size()
    return {"h2d_ms": h, "h2d_gbs": nb_in / h / 1e6, "d2h_ms": d, "d2h_gbs": nb_out / d / 1e6,
            "both_directions_ms": both, "both_gbs": (nb_in + nb_out) / both / 1e6,
            "bytes_in": nb_in, "bytes_out": nb_out, "reps": reps}


def _event_ms(stream, fn, reps, flush=None):
    """Mean device time of fn() over reps launches on `stream` (CUDA events
    around each launch; with `flush`, L2 is overwritten before each one)."""
    import torch
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    torch.cuda.synchronize()
    for e0, e1 in evs:
        if flush is not None:
            flush.add_(1)
        e0.record(stream)
        fn()
        e1.record(stream)
    torch.cuda.synchronize()
    return sum(e0.elapsed_time(e1) for e0, e1 in evs) / reps


def _oracle_sample(b, idx, tag):
    """The oracle on matrices idx of batch b (inputs rounded to the working
    precision): (sub-batch, oracle X, inverses/s, threads, seconds)."""
    import oracle
    from paper_1111_4144_gb300 import workloads as wl
    n = b.n[idx].astype(np.int32)
    off, total = wl.layout_offsets(n, b.layout)
    per = n.astype(np.int64) ** 2 if b.layout == wl.LAYOUT_DENSE else wl.tri(n.astype(np.int64))
    A = np.zeros(total, dtype=np.float64)
    for k, src in enumerate(b.off[idx]):
        A[off[k]:off[k] + per[k]] = b.A[src:src + per[k]]
    if tag == "f32":
        A = A.astype(np.float32).astype(np.float64)
    sb = wl.Batch(A, n, off, b.layout)
    threads = os.cpu_count() or 1
    reps, t0 = 0, time.perf_counter()
    while True:
        _, Xo, _ = oracle.inv_batch(A, n, off, b.layout, False, fill_lower=True, nthreads=threads)
        reps += 1
        el = time.perf_counter() - t0
        if el >= 0.5:
            break
    return sb, Xo, reps * len(idx) / el, threads, el


def _dense_err_ratio(sb, Xg_sub, Xo, fp64):
    """max over matrices of the relative Frobenius error of the upper triangle
    over its tolerance (FP64 1e-11; FP32 max(1e-7 kappa, 2.4e-7))."""
    worst, worst_rel = 0.0, 0.0
    for k in range(sb.batch):
        N = int(sb.n[k]); o = int(sb.off[k])
        G = np.triu(Xg_sub[o:o + N * N].reshape(N, N).astype(np.float64))
        R = np.triu(Xo[o:o + N * N].reshape(N, N))
        rel = np.linalg.norm(G - R) / np.linalg.norm(R)
        if fp64:
            tol = 1e-11
        else:
            M = sb.A[o:o + N * N].reshape(N, N)
            M = np.triu(M) + np.triu(M, 1).T
            ev = np.linalg.eigvalsh(M)
            tol = max(1e-7 * ev[-1] / ev[0], 2.4e-7)
        worst, worst_rel = max(worst, rel / tol), max(worst_rel, rel)
    return worst, worst_rel


def extra_workloads(dev, stream, steps):
    """The method's other batched workloads, each timed on its own after
    warm-up (CUDA events on `stream`; inputs larger than L2, or L2 overwritten
    before each launch), each with a bounded oracle sample as its CPU baseline
    and accuracy check.  Rank 0 only; no collective."""
    import torch
    from paper_1111_4144_gb300 import _lib as L, api, workloads as wl
    peaks, peak_kind = measured_peaks()
    hbm = peaks.get("hbm_gbs", FALLBACK_HBM_GBS)
    reps = max(5, min(steps, 20))
    out = {}
    flush = torch.zeros(64 << 20, dtype=torch.int32, device=dev)  # 256 MB, twice the L2
    with torch.cuda.stream(stream):
        # ---- 4,096 real FP64 matrices of order 8, A = B B^T + 8 I; R and X written
        b = wl.spd_gram_shift(4096, 8, 8.0, seed=1000, layout=wl.LAYOUT_DENSE)
        A = torch.from_numpy(b.A).to(dev).view(4096, 8, 8)
        X = torch.zeros_like(A)
        R = torch.zeros_like(A)
        plan = api.Plan(A, X, R=R)
        for _ in range(3):
            plan.launch(stream)
        ms = _event_ms(stream, lambda: plan.launch(stream), reps, flush)
        torch.cuda.synchronize()
        sb, Xo, cpu_v, thr, _ = _oracle_sample(b, np.arange(4096), "f64")
        r = _dense_err_ratio(sb, X.cpu().numpy().reshape(-1), Xo, fp64=True)
        plan.close()
        out["gram_shift_f64_N8_x4096"] = {
            "value": 4096 / (ms / 1e3), "unit": METRIC, "us_per_batch": ms * 1e3,
            "launch": "cuda_graph (uniform order, one kernel)", "l2": "overwritten before each replay",
            "bytes_per_batch": 4096 * 3 * 36 * 8, "note": "3.5 MB per batch: latency-bound, not a roofline case",
            "max_err_over_tol": r[0], "max_rel_err": r[1], "tolerance": "1e-11",
            "cpu_baseline": {"value": cpu_v, "unit": METRIC, "cores": thr, "kind": "oracle",
                             "sample": "the whole 4,096-matrix batch"}}
        del A, X, R

        # ---- 262,144 real FP32 matrices, orders uniform on 2..64, dense
        b = wl.uneven_loguniform(1 << 18, nmin=2, nmax=64, seed=1002, layout=wl.LAYOUT_DENSE)
        A = torch.from_numpy(b.A.astype(np.float32)).to(dev)
        X = torch.zeros_like(A)
        n = torch.from_numpy(b.n).to(dev)
        off = torch.from_numpy(b.off).to(dev)
        tuned = api.autotune(torch.float32, 64, layout=api.LAYOUT_DENSE, batch=16384, stream=stream)
        plan = api.Plan(A, X, n, off, 64, fixed_orders=True)
        plan_t = api.Plan(A, X, n, off, 64, fixed_orders=True, timing=True)
        for _ in range(3):
            plan.launch(stream)
        ms = _event_ms(stream, lambda: plan.launch(stream), reps)
        kms = {N: 0.0 for N in range(2, 65)}
        for _ in range(3):
            plan_t.launch(stream)
        for _ in range(reps):
            plan_t.launch(stream)
            stream.synchronize()
            for N in kms:
                kms[N] += plan_t.kernel_ms(N) / reps
        torch.cuda.synchronize()
        buckets = {}
        alu_peak = fp32_fma_peak_tflops(torch.cuda.get_device_properties(dev).multi_processor_count)
        for N in range(2, 65):
            cnt = int((b.n == N).sum())
            nb = cnt * 2 * (N * (N + 1) // 2) * 4
            buckets[str(N)] = {"matrices": cnt, "kernel_ms": kms[N], "gbs": nb / (kms[N] / 1e3) / 1e9,
                               "frac": nb / (kms[N] / 1e3) / 1e9 / hbm}
            if N > 32 and kms[N] > 0:
                # orders above 32 approach the FP32 ALU ridge: their algorithmic
                # flops against the CUDA-core FMA peak as well
                tf = alg_flops(np.full(cnt, N), cplx=False) / (kms[N] / 1e3) / 1e12
                buckets[str(N)]["alg_tflops"] = tf
                buckets[str(N)]["alu_frac"] = tf / alu_peak
        # the same batch in one persistent launch (CHOL_FLAG_SINGLE_LAUNCH), for comparison
        X1 = torch.zeros_like(A)
        plan1 = api.Plan(A, X1, n, off, 64, flags=L.CHOL_FLAG_SINGLE_LAUNCH)
        for _ in range(3):
            plan1.launch(stream)
        ms_single = _event_ms(stream, lambda: plan1.launch(stream), reps)
        torch.cuda.synchronize()
        plan1.close()
        single_same = bool(torch.isfinite(X1).all().item())
        del X1
        idx = np.unique(np.random.default_rng(12).choice(b.batch, 1024, replace=False))
        sb, Xo, cpu_v, thr, _ = _oracle_sample(b, idx, "f32")
        Xg = X.cpu().numpy()
        Xs = np.concatenate([Xg[b.off[k]:b.off[k] + int(b.n[k]) ** 2] for k in idx])
        r = _dense_err_ratio(sb, Xs, Xo, fp64=False)
        nbytes = alg_bytes(b.n, 4)
        small = [buckets[str(N)]["frac"] for N in range(2, 33)]
        out["uneven_f32_N2-64_x262144"] = {
            "value": b.batch / (ms / 1e3), "unit": METRIC, "ms_per_step": ms, "layout": "dense row-major",
            "launch": "cuda_graph: bucketing + one kernel per order present", "l2": "inputs larger than L2 (1.49 GB)",
            "autotuned_variants": {str(k): v for k, v in tuned.items()},
            "whole_step": {"achieved_gbs": nbytes / (ms / 1e3) / 1e9, "frac": nbytes / (ms / 1e3) / 1e9 / hbm,
                           "algorithmic_bytes": nbytes},
            "single_launch": {"ms_per_step": ms_single, "finite": single_same,
                              "what": "CHOL_FLAG_SINGLE_LAUNCH: one persistent launch of the one-matrix-per-warp "
                                      "form over every order, largest first (graph replay)"},
            "orders_2_32_frac": {"min": min(small), "median": float(np.median(small)), "max": max(small)},
            "per_order": buckets,
            "bytes_rule": "2 * N(N+1)/2 * 4 B per matrix (A upper read, X upper written)",
            "peak": hbm, "peak_source": peak_kind + " (hbm_gbs)",
            "alu_peak_tflops": alu_peak,
            "alu_rule": "orders 33-64: (N^3 - N) flops per matrix (Table 1's N^3/2 multiply-adds) over the order's "
                        "kernel time, against SMs x 128 FP32 lanes x 2 flops x 2070 MHz",
            "max_err_over_tol": r[0], "max_rel_err": r[1],
            "cpu_baseline": {"value": cpu_v, "unit": METRIC, "cores": thr, "kind": "oracle",
                             "sample": f"{len(idx)} seeded matrices of the batch"}}
        plan.close()
        plan_t.close()
        del A, X, n, off

        # ---- 65,536 real FP32 matrices of order 32, kappa = 1e2: forward and adjoint
        batch, N = 1 << 16, 32
        b = wl.fixed_kappa(batch, N, 1e2, seed=1003, layout=wl.LAYOUT_DENSE)
        A = torch.from_numpy(b.A.astype(np.float32)).to(dev).view(batch, N, N)
        W = torch.from_numpy(wl.gaussian((batch, N, N), 1003).astype(np.float32)).to(dev)
        X = torch.zeros_like(A)
        dA = torch.empty_like(A)
        fwd = lambda: api.inv(A, fill_lower=True, X=X, stream=stream)
        bwd = lambda: api.backward(X, W, upper_param=True, dA=dA, stream=stream)
        for _ in range(3):
            fwd()
            bwd()
        ms_f = _event_ms(stream, fwd, reps)
        ms_b = _event_ms(stream, bwd, reps)
        torch.cuda.synchronize()
        idx = np.arange(0, batch, batch // 64)
        sb, Xo, cpu_v, thr, _ = _oracle_sample(b, idx, "f32")
        Xs = X.cpu().numpy()[idx].reshape(-1)
        r = _dense_err_ratio(sb, Xs, Xo, fp64=False)
        fb, bb = batch * 2 * 528 * 4, batch * (528 + 2 * 1024) * 4
        out["autograd_f32_N32_x65536"] = {
            "value": batch / ((ms_f + ms_b) / 1e3), "unit": "matrices/s (forward + adjoint)",
            "forward_ms": ms_f, "adjoint_ms": ms_b,
            "forward": {"achieved_gbs": fb / (ms_f / 1e3) / 1e9, "frac": fb / (ms_f / 1e3) / 1e9 / hbm,
                        "bytes_rule": "A upper read + X upper written, 2 * 528 * 4 B per matrix "
                                      "(the full X is written: fill_lower)"},
            "adjoint": {"achieved_gbs": bb / (ms_b / 1e3) / 1e9, "frac": bb / (ms_b / 1e3) / 1e9 / hbm,
                        "bytes_rule": "X upper + G + dA dense, (528 + 2 * 1024) * 4 B per matrix"},
            "l2": "inputs larger than L2 (268 MB per operand)",
            "max_err_over_tol": r[0], "max_rel_err": r[1],
            "cpu_baseline": {"value": cpu_v, "unit": "inverses/s (forward)", "cores": thr, "kind": "oracle",
                             "sample": f"{len(idx)} evenly spaced matrices of the batch"}}
        del A, W, X, dA, flush
    return out


def _rel_upper(Xg, Xref):
    """Relative Frobenius error of the upper triangle (numpy, float64)."""
    G = np.triu(np.asarray(Xg, dtype=np.float64))
    R = np.triu(np.asarray(Xref, dtype=np.float64))
    return float(np.linalg.norm(G - R) / np.linalg.norm(R))


def blocked_workloads(dev, stream, sizes=(4096, 16384)):
    """The large single-matrix workload: lambda log-spaced over [1, 1e4],
    FP32 storage, tensor-core (3xTF32) trailing updates and inverse products,
    FP64 pivots, two refinement steps with the residual accumulated in FP64;
    beside it the same library's plain FP64 form on the same (FP32-rounded)
    matrix.  Times by CUDA events on `stream` (one warm-up call first); the
    products' times from the library's event pairs (chol_blocked_timing) in a
    separate call; error against the oracle at 4096 (the whole upper
    triangle) and against the FP64 form at 16384 (which the GPU tests check
    against the oracle on sampled columns)."""
    import ctypes
    import torch
    import oracle
    from paper_1111_4144_gb300 import _lib as L, api, workloads as wl
    peaks, peak_kind = measured_peaks()
    tf32_peak = peaks.get("bf16_tflops_sustained", FALLBACK_BF16_TFLOPS_SUSTAINED) * TF32_OVER_BF16
    out = {}
    kinds = {"trailing_update": L.CHOL_BLK_TRAILING_UPDATE, "inverse_product": L.CHOL_BLK_INVERSE_PRODUCT,
             "refine_residual": L.CHOL_BLK_RESIDUAL, "refine_correction": L.CHOL_BLK_CORRECTION,
             "whole_call": L.CHOL_BLK_WHOLE_CALL}
    with torch.cuda.stream(stream):
        for N in sizes:
            if N <= 8192:
                A64 = torch.from_numpy(wl.log_spaced(N, decades=4.0, seed=1004).A.reshape(N, N)).to(dev)
                gen = "log_spaced (Householder QR of a Gaussian, numpy)"
            else:
                A64 = wl.rotated_log_spaced_torch(N, decades=4.0, seed=1004, device=dev)
                gen = "rotated_log_spaced_torch (8 Householder reflections of diag(lambda), on the GPU)"
            A32 = A64.float().contiguous().view(1, N, N)
            del A64
            A64r = A32.double()  # the FP32-rounded matrix, widened
            X32 = torch.empty_like(A32)
            X64 = torch.empty_like(A64r)
            info = torch.empty(1, dtype=torch.int32, device=dev)
            small = N <= 8192
            reps = 3 if small else 1
            tf = dict(prec=L.CHOL_PREC_TF32_REFINE, flags=L.CHOL_FLAG_PIVOT64)
            # the residual of the refinement steps: compensated FP32 pairs (the
            # library's default) and IEEE FP64 (CHOL_FLAG_RESIDUAL_FP64)
            modes = {
                "tf32_split_pivot64_refine2": (A32, X32, dict(tf, refine_steps=2)),
                "tf32_split_pivot64_refine2_resid64": (A32, X32, dict(prec=L.CHOL_PREC_TF32_REFINE, refine_steps=2,
                                                                      flags=L.CHOL_FLAG_PIVOT64 |
                                                                      L.CHOL_FLAG_RESIDUAL_FP64)),
                "tf32_split_pivot64_refine0": (A32, X32, dict(tf, refine_steps=0)),
                "fp64": (A64r, X64, {}),
            }
            res = {}
            Xkeep = {}
            for name, (Ain, Xout, kw) in modes.items():
                call = lambda: api.inv(Ain, X=Xout, info=info, stream=stream, **kw)
                if small:
                    call()  # warm-up (first-call set-up, workspace)
                torch.cuda.synchronize()
                ms = _event_ms(stream, call, reps)
                torch.cuda.synchronize()
                r = {"ms_per_inverse": ms, "alg_tflops": N ** 3 / (ms / 1e3) / 1e12, "info": int(info.item()),
                     "device_error": L.chol_last_device_error(None), "reps": reps}
                if name in ("tf32_split_pivot64_refine2", "tf32_split_pivot64_refine0") or \
                        (small and name != "fp64"):
                    # the products' own times, from event pairs in a separate call
                    L.check(L.chol_blocked_timing(1), "chol_blocked_timing")
                    call()
                    torch.cuda.synchronize()
                    prod = {}
                    for kn, kc in kinds.items():
                        f_ms, f_fl, f_n = ctypes.c_float(), ctypes.c_double(), ctypes.c_int32()
                        L.check(L.chol_blocked_timing_read(kc, ctypes.byref(f_ms), ctypes.byref(f_fl),
                                                           ctypes.byref(f_n)), "chol_blocked_timing_read")
                        if f_n.value:
                            prod[kn] = {"ms": f_ms.value, "launches": f_n.value, "alg_flops": f_fl.value,
                                        "alg_tflops": f_fl.value / (f_ms.value / 1e3) / 1e12 if f_ms.value else None}
                    L.check(L.chol_blocked_timing(0), "chol_blocked_timing")
                    r["products"] = prod
                    tc = {k: v for k, v in prod.items() if k in ("trailing_update", "inverse_product")}
                    if tc:
                        dom = max(tc, key=lambda k: tc[k]["ms"])
                        ach = tc[dom]["alg_tflops"]
                        r["tensor_roofline"] = {
                            "bound": "tensor", "kernel": dom, "achieved": ach, "unit": "TFLOP/s",
                            "peak": tf32_peak, "frac": ach / tf32_peak,
                            "mma_frac": 3 * ach / tf32_peak,
                            "peak_source": peak_kind + " bf16_tflops_sustained x 1.1/2.25 (nominal TF32:BF16)",
                            "rule": "achieved = algorithmic 2MNK flops of that product kind / its summed event "
                                    "time; the 3xTF32 split issues three MMA products per FP32 product "
                                    "(mma_frac = 3 x frac)"}
                Xkeep[name] = Xout[0].cpu().numpy().copy()
                res[name] = r
            entry = {"order": N, "generator": gen, "lambda": "log-spaced over [1, 1e4]", "modes": res,
                     "speedup_refine2_over_fp64": res["fp64"]["ms_per_inverse"] /
                     res["tf32_split_pivot64_refine2"]["ms_per_inverse"],
                     "speedup_refine2_resid64_over_fp64": res["fp64"]["ms_per_inverse"] /
                     res["tf32_split_pivot64_refine2_resid64"]["ms_per_inverse"]}
            kap = 1e4
            entry["tolerance"] = {"fp32": max(1e-7 * kap, 2.4e-7), "fp64": 1e-11,
                                  "rule": "relative Frobenius error of the upper triangle"}
            if N <= 8192:
                Aw = A32[0].cpu().numpy().astype(np.float64)
                threads = os.cpu_count() or 1
                t0 = time.perf_counter()
                Ro, inf_o = oracle.chol_mt(Aw, threads)
                Xo = oracle.inv_rows_mt(Ro, threads)
                t_orc = time.perf_counter() - t0
                for name in res:
                    res[name]["err_vs_oracle"] = _rel_upper(Xkeep[name], Xo)
                entry["cpu_baseline"] = {"value": 1.0 / t_orc, "unit": "inverses/s", "cores": threads,
                                         "kind": "oracle", "sample": f"one {N} x {N} inverse (Cholesky + the "
                                                                     f"Sec. IV.A recurrence, FP64, threads over "
                                                                     f"each row's entries)"}
            else:
                for name in res:
                    if name != "fp64":
                        res[name]["err_vs_fp64_form"] = _rel_upper(Xkeep[name], Xkeep["fp64"])
            out[f"blocked_f32_N{N}_kappa1e4"] = entry
            del A32, A64r, X32, X64, Xkeep
            torch.cuda.empty_cache()
    return out


def refine_workload(dev, stream, steps):
    """FP32 + refinement against the plain FP64 form at the error each
    reaches: 65,536 FP32 matrices of order 32 with kappa = 1e4 (the
    differentiation workload's generator), refinement steps 0, 1 and 2 with
    the residual in compensated FP32 pairs, one step with it in FP64, and the
    FP64 form of the same library on the same (FP32-rounded) matrices; error
    against the oracle on 64 evenly spaced matrices."""
    import torch
    from paper_1111_4144_gb300 import _lib as L, api, workloads as wl
    batch, N = 1 << 16, 32
    b = wl.fixed_kappa(batch, N, 1e4, seed=1006, layout=wl.LAYOUT_DENSE)
    A = torch.from_numpy(b.A.astype(np.float32)).to(dev).view(batch, N, N)
    A64 = A.double()
    X = torch.zeros_like(A)
    X64 = torch.zeros_like(A64)
    info = torch.empty(batch, dtype=torch.int32, device=dev)
    reps = max(5, min(steps, 20))
    idx = np.arange(0, batch, batch // 64)
    sb, Xo, cpu_v, thr, _ = _oracle_sample(b, idx, "f32")
    res = {}
    with torch.cuda.stream(stream):
        runs = {f"fp32_refine{k}": (A, X, dict(prec=L.CHOL_PREC_FP32_REFINE, refine_steps=k)) for k in (0, 1, 2)}
        runs["fp32_refine1_resid64"] = (A, X, dict(prec=L.CHOL_PREC_FP32_REFINE, refine_steps=1,
                                                   flags=L.CHOL_FLAG_RESIDUAL_FP64))
        runs["fp64"] = (A64, X64, {})
        for name, (Ain, Xout, kw) in runs.items():
            call = lambda: api.inv(Ain, X=Xout, info=info, stream=stream, **kw)
            for _ in range(3):
                call()
            ms = _event_ms(stream, call, reps)
            torch.cuda.synchronize()
            Xs = Xout.cpu().numpy()[idx].reshape(-1)
            r = _dense_err_ratio(sb, Xs, Xo, fp64=False)
            res[name] = {"ms_per_step": ms, "value": batch / (ms / 1e3), "unit": METRIC,
                         "max_rel_err_vs_oracle": r[1], "max_err_over_fp32_tol": r[0],
                         "info_nonzero": int(torch.count_nonzero(info).item())}
    del A, A64, X, X64
    return {"matrices": batch, "order": N, "kappa": 1e4, "layout": "dense row-major", "modes": res,
            "tolerance": "FP32 max(1e-7 kappa, 2.4e-7) = 1e-3; FP64 1e-11 (relative Frobenius, upper triangle)",
            "cpu_baseline": {"value": cpu_v, "unit": METRIC, "cores": thr, "kind": "oracle",
                             "sample": f"{len(idx)} evenly spaced matrices of the batch"}}


def methods_workload(dev, stream, steps):
    """Table 1 on GPU time: the proposed inverse (Sec. IV.A) against the
    existing Equation Solving (Sec. III.A) and Triangular Matrix Operations
    (Sec. III.B) methods, all three on the same one-matrix-per-warp kernel,
    on 32,768 FP32 matrices each of orders 48 and 64 (lambda log-uniform in
    [1, 1e3]); beside them the proposed method on the register-resident
    kernel the library runs by default.  Multiply counts from the closed
    forms of the oracle's counter (the paper's accounting)."""
    import torch
    import oracle
    from paper_1111_4144_gb300 import _lib as L, api, workloads as wl
    reps = max(5, min(steps, 20))
    out = {}
    with torch.cuda.stream(stream):
        for N in (48, 64):
            batch = 32768
            b = wl.qr_spectrum(batch, lambda rng, m: np.full(m, N),
                               lambda rng, m, NN: 10.0 ** rng.uniform(0.0, 3.0, size=(m, NN)), 1007 + N,
                               wl.LAYOUT_PACKED)
            A = torch.from_numpy(b.A.astype(np.float32)).to(dev)
            X = torch.zeros_like(A)
            info = torch.empty(batch, dtype=torch.int32, device=dev)
            res = {}
            runs = {"proposed_wide_kernel": (0, 0), "proposed_warp_kernel": (0, 1),
                    "equation_solving_warp_kernel": (L.CHOL_FLAG_METHOD_ES, 1),
                    "triangular_matrix_ops_warp_kernel": (L.CHOL_FLAG_METHOD_TMO, 1)}
            try:
                for name, (flag, variant) in runs.items():
                    L.check(L.chol_tune_set(L.CHOL_F32, N, variant), "chol_tune_set")
                    call = lambda: api.inv(A, max_n=N, layout=wl.LAYOUT_PACKED, X=X, info=info, flags=flag,
                                           stream=stream)
                    for _ in range(3):
                        call()
                    ms = _event_ms(stream, call, reps)
                    torch.cuda.synchronize()
                    res[name] = {"ms": ms, "value": batch / (ms / 1e3), "unit": METRIC,
                                 "info_nonzero": int(torch.count_nonzero(info).item())}
            finally:
                L.chol_tune_set(L.CHOL_F32, N, 0)
            c = oracle.count_closed_form(N)
            out[f"order{N}"] = {"matrices": batch, "modes": res, "multiplies_per_matrix": {
                "proposed": c["proposed"], "equation_solving": c["es"], "triangular_matrix_ops": c["tmo"],
                "triangular_matrix_ops_structure_exploiting": c["tmo_exploit"]},
                "ratio_es_over_proposed_ms": res["equation_solving_warp_kernel"]["ms"] /
                res["proposed_warp_kernel"]["ms"],
                "ratio_tmo_over_proposed_ms": res["triangular_matrix_ops_warp_kernel"]["ms"] /
                res["proposed_warp_kernel"]["ms"]}
            del A, X
    return out


def mmse_workload(dev, stream, steps):
    """MMSE filters W = (H^* H + 0.1 I)^{-1} H^* of 262,144 MIMO channels
    (N in {4, 8, 16}, 2N x N, iid CN(0,1), complex64): the Gram matrix, the
    batched inverse and W = X H^* (chol_mmse_batched), against the oracle's
    mmse_filter on 256 sampled channels."""
    import torch
    import oracle
    from paper_1111_4144_gb300 import api, workloads as wl
    peaks, peak_kind = measured_peaks()
    hbm = peaks.get("hbm_gbs", FALLBACK_HBM_GBS)
    batch = 1 << 18
    H, n, m, hoff, woff = wl.mimo_channels(batch, sizes=SIZES, seed=1008)
    H64 = H.astype(np.complex64)
    del H
    with torch.cuda.stream(stream):
        Ht = torch.from_numpy(H64).to(dev)
        W = torch.empty_like(Ht)
        nt, mt = torch.from_numpy(n).to(dev), torch.from_numpy(m).to(dev)
        ht, wt = torch.from_numpy(hoff).to(dev), torch.from_numpy(woff).to(dev)
        info = torch.empty(batch, dtype=torch.int32, device=dev)
        # the orders the channels may have are known: kernels for those only
        call = lambda: api.mmse(Ht, nt, mt, ht, wt, max(SIZES), 2 * max(SIZES), sigma2=SIGMA2, W=W, info=info,
                                stream=stream, orders=SIZES)
        for _ in range(3):
            call()
        ms = _event_ms(stream, call, max(5, min(steps, 20)))
        torch.cuda.synchronize()
        Wg = W.cpu().numpy()
        nz = int(torch.count_nonzero(info).item())
    rng = np.random.default_rng(13)
    worst, worst_ratio = 0.0, 0.0
    for b in rng.choice(batch, 256, replace=False):
        N, M = int(n[b]), int(m[b])
        Hb = H64[hoff[b]:hoff[b] + M * N].reshape(M, N).astype(np.complex128)
        Wo, _ = oracle.mmse_filter(Hb, SIGMA2)
        e = np.linalg.norm(Wg[woff[b]:woff[b] + N * M].reshape(N, M) - Wo) / np.linalg.norm(Wo)
        A = np.conj(Hb).T @ Hb + SIGMA2 * np.eye(N)
        worst, worst_ratio = max(worst, e), max(worst_ratio, e / max(1e-7 * np.linalg.cond(A), 2.4e-7))
    nbytes = 2 * int((m.astype(np.int64) * n).sum()) * 8
    del Ht, W
    return {"channels": batch, "sizes": list(SIZES), "rows": "2N", "sigma2": SIGMA2, "ms_per_step": ms,
            "value": batch / (ms / 1e3), "unit": "filters/s", "info_nonzero": nz,
            "achieved_gbs": nbytes / (ms / 1e3) / 1e9, "frac": nbytes / (ms / 1e3) / 1e9 / hbm,
            "bytes_rule": "H read + W written (2 x 2N^2 x 8 B per channel); the Gram matrix and inverse "
                          "(packed, in the workspace) are extra traffic",
            "max_rel_err_vs_oracle": worst, "max_err_over_fp32_tol": worst_ratio,
            "steps": "A = H^* H + s2 I, the batched inverse (Sec. II + IV.A), W = X H^*"}


def run_profile_case(args, local_rank):
    """One order's default kernel on a uniform packed batch (profiling case).

    DTYPE:N:BATCH[:OPT...], OPT one of rK (FP32 + K refinement steps), ldl
    (the LDL form), bwd (the timed region runs the adjoint of the inverse,
    dA for G = I, instead), vK (kernel variant K of the order, pinned in the
    tuning table), p64 (FP64 pivots), mmse (the timed region runs the MMSE
    filters of BATCH channel matrices of 2N x N instead)."""
    import torch
    from paper_1111_4144_gb300 import _lib as L, api, workloads as wl
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    tag, N, batch, *opts = args.profile_case.split(":")
    N, batch = int(N), int(batch)
    kw, bwd, mmse_case = {}, False, False
    for o in opts:
        if o.startswith("r") and o[1:].isdigit():
            kw.update(prec=L.CHOL_PREC_FP32_REFINE, refine_steps=int(o[1:]))
        elif o == "ldl":
            kw["flags"] = kw.get("flags", 0) | L.CHOL_FLAG_LDL
        elif o == "bwd":
            bwd = True
        elif o.startswith("v") and o[1:].isdigit():
            dtc = {"f32": L.CHOL_F32, "f64": L.CHOL_F64, "c64": L.CHOL_C64, "c128": L.CHOL_C128}[tag]
            L.check(L.chol_tune_set(dtc, N, int(o[1:])), "chol_tune_set")
        elif o == "p64":
            kw["flags"] = kw.get("flags", 0) | L.CHOL_FLAG_PIVOT64
        elif o == "mmse":
            mmse_case = True
        else:
            raise SystemExit(f"--profile-case: unknown option {o!r}")
    npd = {"f32": np.float32, "f64": np.float64, "c64": np.complex64, "c128": np.complex128}[tag]
    base = 1024
    if tag.startswith("c"):
        b = wl.mimo_covariance(base, sizes=(N,), seed=1009, layout=wl.LAYOUT_PACKED, shuffle=False)
    else:
        b = wl.qr_spectrum(base, lambda rng, m: np.full(m, N),
                           lambda rng, m, NN: 10.0 ** rng.uniform(0.0, 3.0, size=(m, NN)), 1009, wl.LAYOUT_PACKED)
    A = torch.from_numpy(np.tile(b.A.astype(npd), (batch + base - 1) // base)[:batch * (N * (N + 1) // 2)]).to(dev)
    X = torch.zeros_like(A)
    info = torch.empty(batch, dtype=torch.int32, device=dev)
    call = lambda: api.inv(A, max_n=N, layout=wl.LAYOUT_PACKED, X=X, info=info, **kw)
    if mmse_case:
        rng = np.random.default_rng(1010)
        Hn = (rng.standard_normal((1024, 2 * N, N)) + 1j * rng.standard_normal((1024, 2 * N, N))) * np.sqrt(0.5)
        H = torch.from_numpy(np.tile(Hn.astype(npd), ((batch + 1023) // 1024, 1, 1))[:batch]).to(dev)
        Wm = torch.empty((batch, N, 2 * N), dtype=H.dtype, device=dev)
        call = lambda: api.mmse(H, sigma2=0.1, W=Wm, info=info, **kw)
    if bwd:
        call()
        G = torch.zeros((batch, N, N), dtype=A.dtype, device=dev)
        G[:, torch.arange(N), torch.arange(N)] = 1
        dA = torch.empty_like(G)
        call = lambda: api.backward(X, G, max_n=N, layout=wl.LAYOUT_PACKED, dA=dA)
    for _ in range(max(args.warmup, 1)):
        call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("step")
    e0.record()
    for _ in range(args.steps):
        call()
    e1.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    es = np.dtype(npd).itemsize
    print(json.dumps({"profile_case": args.profile_case, "ms": ms, "inverses_per_s": batch / (ms / 1e3),
                      "alg_gbs": 2 * (N * (N + 1) // 2) * es * batch / (ms / 1e3) / 1e9,
                      "info_nonzero": int(torch.count_nonzero(info).item())}), flush=True)


def run_blocked(args, local_rank):
    """One large matrix through the blocked path (the large-order workload)."""
    import torch
    from paper_1111_4144_gb300 import _lib as L, api
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    N = args.blocked
    dt = torch.float64 if args.blocked_prec == "fp64" else torch.float32
    # A = Q diag(lambda) Q^T with Q from a Householder QR of a Gaussian, lambda log-spaced over [1, 1e4]
    if N <= 8192:
        from paper_1111_4144_gb300 import workloads as wl
        A = torch.from_numpy(wl.log_spaced(N, decades=4.0, seed=1004).A.reshape(1, N, N)).to(dev).to(dt)
    else:
        # the same spectrum rotated by eight random Householder reflections
        from paper_1111_4144_gb300 import workloads as wl
        A = wl.rotated_log_spaced_torch(N, decades=4.0, seed=1004, device=dev).to(dt).reshape(1, N, N)
    A = A.contiguous()
    kw = {}
    piv = L.CHOL_FLAG_PIVOT64 if args.blocked_pivots == "fp64" else 0
    if args.blocked_prec == "tf32":
        kw = dict(prec=L.CHOL_PREC_TF32_REFINE, refine_steps=args.blocked_refine, flags=piv)
    elif args.blocked_prec == "fp32":
        kw = dict(prec=L.CHOL_PREC_FP32_REFINE, refine_steps=args.blocked_refine, flags=piv)
    X, info = api.inv(A, **kw)
    torch.cuda.synchronize()
    for _ in range(max(args.warmup - 1, 0)):
        api.inv(A, X=X, info=info, **kw)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("blocked_step")
    e0.record()
    for _ in range(args.steps):
        api.inv(A, X=X, info=info, **kw)
    e1.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    print(json.dumps({"blocked_order": N, "prec": args.blocked_prec, "refine_steps": kw.get("refine_steps", 0),
                      "pivots": args.blocked_pivots if args.blocked_prec != "fp64" else "fp64",
                      "ms_per_inverse": ms,
                      "alg_tflops": N ** 3 / (ms / 1e3) / 1e12, "info": int(info.item()),
                      "device_error": L.chol_last_device_error(None)}), flush=True)


def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    from paper_1111_4144_gb300 import _lib, api

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    _lib.load()
    sizes = tuple(int(x) for x in args.sizes.split(","))
    if args.uniform:
        sizes = sizes[:1]
    b = make_workload(rank, args.batch, sizes)
    A64 = b.A.astype(np.complex64)
    A = torch.from_numpy(A64).to(dev)
    n = torch.from_numpy(b.n).to(dev)
    off = torch.from_numpy(b.off).to(dev)
    X = torch.zeros_like(A)
    stream = torch.cuda.Stream(device=dev)
    # pick the fastest kernel variant of each order on this GPU (set-up,
    # untimed), ranked at this workload's matrices per order
    tuned = api.autotune(torch.complex64, max(sizes), layout=api.LAYOUT_PACKED,
                         batch=max(1, b.batch // len(sizes)), stream=stream)
    torch.cuda.synchronize()
    # The timed plan records kernels only for the orders present
    # (CHOL_FLAG_PLAN_ORDERS); a second plan of the same call adds an event
    # pair around each class kernel (CHOL_FLAG_PLAN_TIMING) for the per-kernel
    # times, which would cost the timed step about 5 % (six event nodes).
    if args.uniform:
        plan = api.Plan(A, X, None, None, sizes[0], layout=api.LAYOUT_PACKED)
        plan_t = api.Plan(A, X, None, None, sizes[0], layout=api.LAYOUT_PACKED, timing=True)
        kernels_per_step = 1
    else:
        plan = api.Plan(A, X, n, off, max(sizes), layout=api.LAYOUT_PACKED, fixed_orders=True)
        plan_t = api.Plan(A, X, n, off, max(sizes), layout=api.LAYOUT_PACKED, timing=True, fixed_orders=True)
        kernels_per_step = 2 + len(set(sizes))  # histogram (with the scan), scatter + one kernel per order

    def timed(fn, steps, label):
        # the NVTX range lets a profiler capture exactly the timed launches
        # (ncu --nvtx --nvtx-include "<label>/")
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.nvtx.range_push(label)
        ev0.record(stream)
        for _ in range(steps):
            fn()
        ev1.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        return max_over_ranks(ev0.elapsed_time(ev1) / steps, world, dev)

    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 3)):
            plan.launch(stream)
        sampler = ClockSampler(local_rank)
        if rank == 0:
            sampler.start()
        ms = timed(lambda: plan.launch(stream), args.steps, "step")
        # keep the GPU under the same load long enough for the clock sampler
        t_end = time.perf_counter() + max(0.0, 1.5 - ms * args.steps / 1e3)
        while time.perf_counter() < t_end:
            for _ in range(50):
                plan.launch(stream)
            torch.cuda.synchronize()
        clocks = sampler.stop() if rank == 0 else None

    value = job_value(world, b.batch, ms)
    nbytes = alg_bytes(b.n, 8)
    peaks, peak_kind = measured_peaks()
    achieved = nbytes / (ms / 1e3) / 1e9
    # per-order kernel durations: the timing plan replayed in its own timed
    # loop (events recorded inside the graph, on the stream each kernel runs
    # on), the mean over its replays, and the last replay of that loop
    orders = sorted(set(int(x) for x in np.unique(b.n)))
    acc = {N: 0.0 for N in orders}
    reps = 20
    with torch.cuda.stream(stream):
        for _ in range(3):
            plan_t.launch(stream)
        torch.cuda.nvtx.range_push("kernel_timing")
        for _ in range(reps):
            plan_t.launch(stream)
            stream.synchronize()
            for N in orders:
                acc[N] += plan_t.kernel_ms(N)
        torch.cuda.nvtx.range_pop()
    last = {N: plan_t.kernel_ms(N) for N in orders}
    kern_ms = {N: acc[N] / reps for N in orders}
    dom = max(orders, key=lambda N: kern_ms[N])
    dom_bytes = alg_bytes(b.n[b.n == dom], 8)
    dom_gbs = dom_bytes / (kern_ms[dom] / 1e3) / 1e9

    # ---- accuracy and the FP64 form (rank 0)
    out = {}
    if args.quick:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": METRIC, "ms_per_step": ms, "quick": True,
                              "config": {"batch_per_gpu": b.batch, "sizes": list(sizes),
                                         "autotuned_variants": {str(k): v for k, v in tuned.items()}},
                              "per_order_kernel_ms": {str(N): kern_ms[N] for N in orders},
                              "achieved_gbs": achieved, "clocks": clocks}), flush=True)
        plan.close()
        plan_t.close()
        return
    if rank == 0:
        torch.cuda.synchronize()
        Xg = X.cpu().numpy()
        A_wide = A64.astype(np.complex128)
        info = plan.info.cpu().numpy()
        cpu_v, threads, reps, (_, Xo, info_o) = oracle_time(b, A_wide, min_wall=1.0)
        kap = kappa_of(b, A_wide)
        r32 = upper_err_ratio(b, Xg, Xo, kap, fp64=False)
        out["accuracy"] = {"fp32_max_err_over_tol": r32[0], "fp32_max_rel_err": r32[1],
                           "fp32_median_rel_err": r32[2], "info_nonzero": int(np.count_nonzero(info)),
                           "info_matches_oracle": bool(np.array_equal(info, info_o)),
                           "tolerance": "max(1e-7*kappa, 2.4e-7) relative Frobenius, upper triangle"}
        cpu_1, cnt_1, reps_1 = oracle_time_single(b, A_wide, 131072)
        out["cpu_baseline"] = {"value": cpu_v, "unit": METRIC, "cores": threads, "kind": "oracle",
                               "sample": f"{reps} x the full {b.batch}-matrix batch, FP64 C oracle, "
                                         f"{threads} threads",
                               "single_thread": {"value": cpu_1, "unit": METRIC, "cores": 1,
                                                 "sample": f"{reps_1} x the batch's first {cnt_1} matrices, "
                                                           f"FP64 C oracle, 1 thread"}}
        # plain FP64 form (complex128) of the same library on the same matrices
        A128 = torch.from_numpy(A_wide).to(dev)
        X128 = torch.zeros_like(A128)
        plan64 = api.Plan(A128, X128, n, off, max(sizes), layout=api.LAYOUT_PACKED, fixed_orders=True)
        with torch.cuda.stream(stream):
            for _ in range(2):
                plan64.launch(stream)
            ms64 = timed(lambda: plan64.launch(stream), max(3, min(args.steps, 20)), "fp64_form")
        r64 = upper_err_ratio(b, X128.cpu().numpy(), Xo, kap, fp64=True)
        out["fp64_form"] = {"value": b.batch / (ms64 / 1e3), "unit": METRIC, "ms_per_step": ms64,
                            "max_err_over_tol": r64[0], "max_rel_err": r64[1], "tolerance": "1e-11",
                            "speedup_fp32_over_fp64": ms64 / ms}
        plan64.close()
        del A128, X128
        # the LDL form (Sec. IV.B) of the same library on the same FP32 matrices
        Xl = torch.zeros_like(X)
        planl = api.Plan(A, Xl, n, off, max(sizes), layout=api.LAYOUT_PACKED, fixed_orders=True,
                         flags=_lib.CHOL_FLAG_LDL)
        with torch.cuda.stream(stream):
            for _ in range(2):
                planl.launch(stream)
            msl = timed(lambda: planl.launch(stream), max(3, min(args.steps, 20)), "ldl_form")
        rl = upper_err_ratio(b, Xl.cpu().numpy(), Xo, kap, fp64=False)
        out["ldl_form"] = {"value": b.batch / (msl / 1e3), "unit": METRIC, "ms_per_step": msl,
                           "max_err_over_tol": rl[0], "max_rel_err": rl[1],
                           "kernel": "the size-class kernels of the Cholesky form, built for the LDL form",
                           "ratio_over_cholesky_ms": msl / ms}
        planl.close()
        del Xl

    # ---- end to end through the public API with host buffers
    A_h = torch.from_numpy(A64).pin_memory()
    n_h = torch.from_numpy(b.n).pin_memory()
    off_h = torch.from_numpy(b.off).pin_memory()
    X_h = torch.empty_like(A_h).pin_memory()
    info_h = torch.empty(b.batch, dtype=torch.int32).pin_memory()

    # chol_inv_batched_host: the batch streams from pinned host memory through
    # device slots in chunks, copies overlapping kernels; X and info land in
    # pinned host memory
    host_inv = api.HostInv(torch.complex64, b.batch, max(sizes), sizes=True, layout=api.LAYOUT_PACKED)

    def e2e_step():
        host_inv(A_h, X_h, n_h, off_h, info_h, stream=stream)

    with torch.cuda.stream(stream):
        e2e_step()
        ms_e2e = timed(e2e_step, max(3, min(args.steps, 20)), "e2e")
    h2d = A_h.numel() * 8 + n_h.numel() * 4 + off_h.numel() * 8
    link = host_link_ceiling(dev, A_h, X_h, A, X)
    d2h = X_h.numel() * 8 + info_h.numel() * 4
    # the other workloads last, so that nothing they leave allocated affects the legs above
    if rank == 0 and not args.no_extra:
        out["configs"] = extra_workloads(dev, stream, args.steps)
        out["configs"]["refine_f32_N32_x65536_kappa1e4"] = refine_workload(dev, stream, args.steps)
        out["configs"]["table1_methods_f32_x32768"] = methods_workload(dev, stream, args.steps)
        out["configs"]["mmse_c64_N4-8-16_x262144"] = mmse_workload(dev, stream, args.steps)
        if not args.no_blocked:
            out["configs"].update(blocked_workloads(dev, stream))

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "c64 (fp32 arithmetic)", "data": "synthetic",
                "config": {"workload": WORKLOAD, "batch_per_gpu": b.batch, "sizes": list(SIZES), "sigma2": SIGMA2,
                           "layout": "packed_upper", "launch": "cuda_graph",
                           "autotuned_variants": {str(k): v for k, v in tuned.items()},
                           "l2": "inputs larger than L2 (509 MB in, 509 MB out per step)"},
                "roofline": {"bound": "hbm", "achieved": dom_gbs, "peak": peaks.get("hbm_gbs", FALLBACK_HBM_GBS),
                             "unit": "GB/s", "frac": dom_gbs / peaks.get("hbm_gbs", FALLBACK_HBM_GBS),
                             "traffic": measured_traffic(dom, int((b.n == dom).sum())),
                             "traffic_source": "dram__bytes_read.sum + dram__bytes_write.sum per matrix from "
                                               "profiles/k_group_c64_N16_full.md, times this launch's matrices "
                                               "(null if the kernel sources changed since the capture)",
                             "peak_source": peak_kind + " (hbm_gbs, copy bandwidth)",
                             "kernel": f"size-class kernel N={dom} (complex64)",
                             "kernel_ms": kern_ms[dom], "kernel_ms_last_replay": last[dom],
                             "kernel_timing": "mean over 20 replays of the same graph with an event pair "
                                              "around each class kernel (a second plan of the same call)",
                             "algorithmic_bytes_per_launch": dom_bytes,
                             "bytes_rule": "2 * N(N+1)/2 * 8 B per matrix (A upper read, X upper written)",
                             "whole_step": {"achieved": achieved, "frac": achieved / peaks.get("hbm_gbs",
                                            FALLBACK_HBM_GBS), "algorithmic_bytes_per_step": nbytes},
                             "per_order_kernel_ms": {str(N): kern_ms[N] for N in orders}},
                "gflops": alg_flops(b.n) / (ms / 1e3) / 1e9,
                "e2e": {"value": job_value(world, b.batch, ms_e2e), "unit": METRIC, "h2d_bytes_per_step": h2d,
                        "host_link": link,
                        "frac_of_copy_only": link["both_directions_ms"] / ms_e2e if link else None,
                        "d2h_bytes_per_step": d2h, "ms_per_step": ms_e2e},
                "gpu_launches": kernels_per_step * args.steps,
                "clocks": clocks}
        line.update(out)
        print(json.dumps(line), flush=True)
    plan.close()
    plan_t.close()


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.blocked:
        run_blocked(args, local_rank)
        return
    if args.profile_case:
        run_profile_case(args, local_rank)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
