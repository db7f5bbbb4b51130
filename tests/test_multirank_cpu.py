"""The multi-GPU bench path on CPU: two gloo ranks, each with its own shard.

bench.py shards the benchmark batch by rank (weak scaling, no collective on the
data path) and reports the slowest rank's step time; these tests run that
host-side logic in two processes on the gloo backend.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    b = bench.make_workload(rank, batch=64, sizes=(4, 8, 16))
    again = bench.make_workload(rank, batch=64, sizes=(4, 8, 16))
    ms_local = 1.0 + rank  # rank 1 is the slow one
    ms = bench.max_over_ranks(ms_local, world, "cpu")
    value = bench.job_value(world, b.batch, ms)
    np.savez(os.path.join(out_dir, f"r{rank}.npz"), A=b.A, n=b.n, again=again.A, ms=ms, value=value)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_ranks_shard_and_take_the_slowest(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    r = [np.load(tmp_path / f"r{k}.npz") for k in range(world)]
    # each rank's shard is deterministic and different from the other rank's
    for k in range(world):
        assert np.array_equal(r[k]["A"], r[k]["again"])
    assert not np.array_equal(r[0]["A"], r[1]["A"])
    # same shape of work on every rank (weak scaling)
    assert np.array_equal(np.sort(r[0]["n"]), np.sort(r[1]["n"]))
    # every rank reports the slowest rank's time, and the job value counts all ranks' matrices
    for k in range(world):
        assert float(r[k]["ms"]) == 2.0
        assert float(r[k]["value"]) == pytest.approx(world * 64 / 2e-3)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.job_value(1, 1000, 2.0) == pytest.approx(500000.0)


@pytest.mark.timeout(300)
def test_reference_arm_under_torchrun_prints_once():
    """`bench.py --impl reference` launched as two torchrun ranks: rank 0 times
    the oracle and prints the one JSON line, the other rank exits 0 without
    work."""
    import json
    import subprocess
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0",
           "--batch", "3000"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=280)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["config"]["batch"] == 3000
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0
