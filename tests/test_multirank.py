"""The multi-GPU path is replicas only (every rank converts its own batch, nothing is exchanged
on the data path); its host logic -- per-rank inputs, the max-over-ranks job time, rank-0-only
reporting -- runs here as two gloo ranks on the CPU."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    import workloads
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # replicas: each rank's batch comes from its own seed
    alpha = workloads.coefficients(64, 2, decay=0.5, seed=rank)
    # rank r reports (r + 1) * 10 ms for 3 steps of 1000 units
    value, total = bench.job_throughput(10.0 * (rank + 1), 1000, 3, world, dist, device="cpu")
    q.put((rank, float(alpha[0, 0]), value, total))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_timing_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks see the slowest rank's time; the value counts every rank's units
    assert [o[3] for o in out] == [20.0, 20.0]
    assert all(abs(o[2] - 2 * 1000 * 3 / 0.020) < 1e-6 for o in out)
    # different inputs per rank (independent replicas)
    assert out[0][1] != out[1][1]


def test_reference_arm_nonzero_rank_exits_quietly():
    """Under torchrun only rank 0 times and prints the oracle arm; other ranks exit 0."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "1"], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_reference_arm_line_contract():
    """The oracle arm prints one JSON line with the keys the bench contract asks for (runs on
    the host cores, no GPU)."""
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "1"], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e", "impl"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["warmup"] >= 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"]
