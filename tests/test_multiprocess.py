"""The N > 1 path of bench.py on CPU processes with the gloo backend (world size 2).

Every run of the library uses one GPU, so N > 1 runs N independent replicas of the
workload (weak scaling): the ranks meet only at a barrier before and after the timed
region and in one max-reduction of the measured time; rank 0 alone prints.  These tests
run that host logic with gloo on the CPU (no GPU), including the CPU reference arm under
torch.distributed.run.
"""

import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, queue):
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    r, local, w = bench.dist_setup("gloo")
    bench.barrier(w)
    t = bench.max_over_ranks(1.5 + r, w)  # each rank "measured" a different time
    bench.barrier(w)
    queue.put((r, local, w, t))
    dist.destroy_process_group()


def test_replica_timing_takes_the_max_over_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[2] == 2 for o in out)
    assert all(o[3] == 2.5 for o in out)  # both ranks see the slowest rank's time


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    env = dict(os.environ)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        os.environ.pop(k, None)
    try:
        assert bench.dist_setup("gloo") == (0, 0, 1)
        assert bench.max_over_ranks(3.0, 1) == 3.0
    finally:
        os.environ.clear()
        os.environ.update(env)


@pytest.mark.timeout(300)
def test_reference_arm_under_torchrun_prints_once():
    """bench.py --impl reference with two ranks: rank 0 times the oracle and prints one JSON
    line, rank 1 exits 0 without work."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--cpu-sample", "512"]
    r = subprocess.run(cmd, capture_output=True, text=True, cwd=ROOT, timeout=280)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"


@pytest.mark.timeout(300)
def test_reference_arm_json_contract():
    """One process: the reference arm prints one JSON line with every key of the benchmark
    contract, the same workload as the GPU arm, and an e2e object with no host transfers."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1", "--cpu-sample", "256"], capture_output=True, text=True, cwd=ROOT, timeout=280)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 1
    assert d["higher_is_better"] is True and d["value"] > 0 and d["unit"] == d["e2e"]["unit"]
    assert d["config"]["workload"].startswith("coupled_spins_d16") and d["config"]["n_steps"] == 1 << 20
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["cpu_baseline"]["value"] == d["value"] and d["cpu_baseline"]["cores"] >= 1


def test_parallel_oracle_timing_matches_the_oracle():
    """The CPU baseline cuts the sample into contiguous slice ranges run by separate oracle
    processes; the ordered product of their partial products is the oracle's U."""
    import numpy as np

    sys.path.insert(0, ROOT)
    import bench
    import oracle
    from paper_2108_07126_gb300 import workloads as wl

    n = 600
    o = bench.time_oracle(n, workers=4)
    prob = wl.coupled_spins(n_steps=n)
    R = oracle.propagate(prob.H0, prob.Hk, prob.c, prob.dt, prob.integrator)
    assert o["cores"] == 4 and o["n"] == n and o["seconds"] > 0 and o["one_core_rate"] > 0
    assert np.max(np.abs(o["U"] - R)) <= 1e-12
