#!/usr/bin/env python3
"""Benchmark: time steps per second to the full propagator U(T) on one GB300.

Workload (default): four coupled spin-1/2 (d = 16), eight controls, fourth-order
Gauss-Legendre Magnus exponent, N = 2^20 slices, complex64 compute (the FP32
path), timed next to the plain FP64 GPU path on the same inputs.  One
"step" = one full propagation (every slice assembled, exponentiated and
multiplied into U(T)) = one kernel launch.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  With --impl reference the FP64 CPU oracle is timed
instead, on a bounded sample of the same workload, on the host cores.
For N > 1 (torchrun) every rank propagates its own copy of the workload
(independent replicas, weak scaling); the timed region is bracketed by
barriers and the slowest rank's time counts.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "time steps/sec to full U(T), by dim, vs plain FP64 GPU path at stated error"
UNIT = "time steps/s"
SM_COUNT, FP32_LANES, FP64_FMA_PER_SM_CLK = 152, 128, 2
L2_FLUSH_BYTES = 256 << 20
# dram__bytes_read.sum + dram__bytes_write.sum of fused_small_kernel<float, 16, GL4> from one ncu capture of
# 2^18 slices (16 921 344 + 0 bytes), scaled per slice: the traffic is the control samples, linear in N
TRAFFIC_BYTES_PER_SLICE = 16917504 / 262144


def _measured_peaks() -> dict:
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


PEAKS = _measured_peaks()
# rates measured on this GPU by parament_measure_peaks (filled once per run, rank 0)
MEASURED = {}


def measure_peaks(b, device: int) -> dict:
    MEASURED.update(b.parament_measure_peaks(device))
    return dict(MEASURED)


def roofline_alu(achieved: float, pipe: str) -> dict:
    """Roofline of a CUDA-core kernel against the measured FMA rate of its pipe (fp32 / fp64)."""
    pk = MEASURED.get(f"{pipe}_tflops_max_clock") or MEASURED.get(f"{pipe}_tflops")
    if pk:
        note = (f"measured {pipe.upper()} FMA rate (parament_measure_peaks: independent FMA chains filling every "
                f"SM, flops per SM clock cycle x the {MEASURED.get('max_sm_clock_mhz', 0):.0f} MHz maximum clock)")
    else:
        per_clk = FP32_LANES if pipe == "fp32" else FP64_FMA_PER_SM_CLK
        pk = SM_COUNT * per_clk * 2 * 2.07e9 / 1e12
        note = "derived from unit counts (measurement unavailable)"
    return {"bound": "alu", "pipe": pipe, "achieved": achieved, "peak": pk, "unit": "TFLOP/s",
            "frac": achieved / pk, "peak_note": note}


def tensor_peak(fmt: str) -> tuple[float, str]:
    """Dense tcgen05 rate of the format (tf32 / bf16): measured here, else the pool's cuBLAS bf16 figure."""
    pk = MEASURED.get(f"{fmt}_tflops")
    if pk:
        return pk, f"measured dense tcgen05 {fmt.upper()} rate (parament_measure_peaks: M128 N256 MMA stream per SM)"
    bf = PEAKS.get("bf16_tflops", 1900.0)
    return (bf * 1.1 / 2.25 if fmt == "tf32" else bf), "cuBLAS bf16 burst of MEASURED_PEAKS.json (TF32 x 1.1 / 2.25)"
TRAFFIC_NOTE = "ncu capture of 2^18 slices (16.92 MB) scaled to the launch; algorithmic 64 B per slice"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n-steps", type=int, default=1 << 20, help="slices of the workload")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--cpu-sample", type=int, default=1 << 16, help="slices in the timed oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the secondary workloads")
    ap.add_argument("--scaling", action="store_true",
                    help="re-run the paper's performance experiments (run time vs d and vs N, CPU crossover) "
                         "instead of the benchmark line")
    ap.add_argument("--scaling-out", default=os.path.join(ROOT, "results", "scaling_sec5.jsonl"),
                    help="file that --scaling writes its JSON lines to (replaced)")
    ap.add_argument("--scaling-report", action="store_true",
                    help="print the markdown tables of a --scaling record (--scaling-out) and exit")
    return ap.parse_args()


def dist_setup(backend):
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend)
    return rank, local, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- clocks


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.proc = None
        self.path = None
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", gpu_id, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 8:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- oracle (CPU baseline)

_ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import numpy as np
import oracle
from paper_2108_07126_gb300 import workloads as wl
prob = wl.coupled_spins(n_steps={n})
per = 1 if prob.integrator == "midpoint" else 2
c = np.ascontiguousarray(prob.c[:, per * {a}:per * {b}])
t0 = time.perf_counter()
for _ in range({reps}):
    U = oracle.propagate(prob.H0, prob.Hk, c, prob.dt, prob.integrator)
dt = time.perf_counter() - t0
np.save({out!r}, U)
print(json.dumps({{"seconds": dt, "reps": {reps}, "n": {b} - {a}}}))
"""


def time_oracle(n_sample: int, reps: int = 1, workers: int = 0) -> dict:
    """Time the FP64 oracle on the first n_sample slices of the workload.

    The slices are cut into `workers` contiguous ranges (default: every host core), each
    propagated by the oracle, unchanged, in its own fresh single-threaded process; the partial
    products are then multiplied in time order.  The parallel time is the slowest worker's
    compute time (process start-up and imports excluded) plus the final products; the per-core
    rate is the workers' mean rate while all of them run.
    """
    import tempfile

    import numpy as np

    workers = max(1, min(workers or (os.cpu_count() or 1), n_sample))
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = "1"
    cuts = [n_sample * w // workers for w in range(workers + 1)]
    with tempfile.TemporaryDirectory() as tmp:
        procs = []
        for w in range(workers):
            out = os.path.join(tmp, f"part{w}.npy")
            code = _ORACLE_SNIPPET.format(root=ROOT, n=n_sample, a=cuts[w], b=cuts[w + 1], reps=reps, out=out)
            procs.append((subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE,
                                           stderr=subprocess.PIPE, text=True, env=env), out))
        res, parts = [], []
        for pr, out in procs:
            so, se = pr.communicate()
            if pr.returncode != 0:
                raise RuntimeError(se)
            res.append(json.loads(so.strip().splitlines()[-1]))
            parts.append(np.load(out))
    t0 = time.perf_counter()
    U = parts[0]
    for P in parts[1:]:
        U = P @ U  # later slices on the left
    t_comb = time.perf_counter() - t0
    seconds = max(r["seconds"] for r in res) / reps + t_comb
    return {"seconds": seconds, "n": n_sample, "cores": workers, "U": U,
            "one_core_rate": statistics.mean(r["n"] * r["reps"] / r["seconds"] for r in res)}


def run_reference(args):
    rank, _, world = dist_setup("gloo")
    if rank != 0:
        return
    n = min(args.cpu_sample, 1 << 16)
    per, one = [], []
    for i in range(args.warmup + args.steps):
        o = time_oracle(n)
        if i >= args.warmup:
            per.append(o["seconds"])
            one.append(o["one_core_rate"])
    ms = 1e3 * statistics.mean(per)
    value = n / (ms * 1e-3)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args.n_steps, "fp64"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": o["cores"], "kind": "oracle",
                         "per_core_value": statistics.mean(one),
                         "sample": f"first {n} slices of the workload per step (FP64 eigendecomposition oracle), "
                                   f"cut into {o['cores']} contiguous ranges, one single-threaded process each"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def workload_config(n_steps, prec):
    return {"workload": f"coupled_spins_d16_magnus4_gl2_N{n_steps}", "dim": 16, "n_steps": n_steps, "n_ctrl": 8,
            "n_coefficients": 45, "integrator": "magnus4_gl2", "precision": prec,
            "l2": f"flushed by a {L2_FLUSH_BYTES >> 20} MiB write between timed steps"}


# ---------------------------------------------------------------- GPU arm


def flops_per_launch(st: dict) -> float:
    """Algorithmic flops of one propagation: assembly + complex d x d products.

    Assembly: 2 flops per (basis matrix, packed real entry): 2 * n_basis * d^2 per slice.
    Each complex d x d product: 8 d^3 flops (Taylor/Paterson-Stockmeyer, squarings, tree).
    """
    d = st["dim"]
    return 2.0 * st["n_basis"] * d * d * st["n_steps"] + 8.0 * d ** 3 * (st["exp_products"] + st["tree_products"])


def time_launches(torch, fn, steps, warmup, flush):
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    evs = []
    for _ in range(steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def batched_sample(probs):
    """Instances of the batched sweep compared with the oracle: the longest of every dimension and
    eight drawn with a fixed seed."""
    import numpy as np

    picked = set()
    for d in sorted({p.dim for p in probs}):
        picked.add(max((i for i, p in enumerate(probs) if p.dim == d), key=lambda i: probs[i].n_steps))
    rng = np.random.default_rng(20210816)
    picked.update(int(i) for i in rng.choice(len(probs), 8, replace=False))
    return sorted(picked)


def secondary_workloads(torch, b, wl, dev, flush, steps=10, warmup=3):
    """Rabi qubit (d = 2, N = 2^14, latency-bound) and the optimal-control gradient (d = 8, N = 65536)."""
    import numpy as np

    import oracle

    out = {}
    prop = b.Propagator(dev.index or 0)
    prob = wl.rabi_qubit()
    for prec, cdt, rdt in (("fp64", torch.complex128, torch.float64), ("fp32", torch.complex64, torch.float32)):
        prop.set_hamiltonians(torch.as_tensor(prob.H0).to(cdt), torch.as_tensor(prob.Hk).to(cdt), prob.integrator)
        prop.set_controls(torch.as_tensor(prob.c).to(rdt).to(dev), prob.dt, prob.n_steps)
        U = torch.empty(2, 2, dtype=cdt, device=dev)
        per = time_launches(torch, lambda: prop.propagate(prec, out=U), steps, warmup, flush)
        ref = oracle.propagate(prob.H0, prob.Hk, prob.c, prob.dt, prob.integrator)
        err = float(np.max(np.abs(U.cpu().numpy().astype(np.complex128) - ref)))
        ms = statistics.mean(per)
        out[f"rabi_qubit_d2_N16384_{prec}"] = {"steps_per_s": prob.n_steps / (ms * 1e-3), "ms_per_step": ms,
                                                "max_abs_err_vs_oracle": err, "launches_per_step": 1}
    prob = wl.gradient_qubits()
    l_ref, g_ref, _ = oracle.loss_and_gradient(prob.H0, prob.Hk, prob.c, prob.dt, prob.V)
    for prec, cdt, rdt in (("fp64", torch.complex128, torch.float64), ("fp32", torch.complex64, torch.float32)):
        prop.set_hamiltonians(torch.as_tensor(prob.H0).to(cdt), torch.as_tensor(prob.Hk).to(cdt), "midpoint")
        prop.set_controls(torch.as_tensor(prob.c).to(rdt).to(dev), prob.dt, prob.n_steps)
        V = torch.as_tensor(prob.V).to(cdt).to(dev)
        res = {}

        def step():
            res["lg"] = prop.propagate_grad(V, prec)

        per = time_launches(torch, step, max(3, steps // 2), 2, flush)
        loss, grad = res["lg"]
        g = grad.cpu().numpy().astype(np.float64)
        ms = statistics.mean(per)
        out[f"gradient_qubits_d8_N65536_{prec}"] = {
            "steps_per_s": prob.n_steps / (ms * 1e-3), "ms_per_step": ms,
            "loss_abs_err_vs_oracle": abs(loss - l_ref),
            "grad_max_rel_err_vs_oracle": float(np.max(np.abs(g - g_ref)) / np.max(np.abs(g_ref))),
            "launches_per_step": 5, "timing": "host wall clock incl. the loss read-back"}
    # ---- batched sweep: 256 instances, d in {2..64}, N log-uniform in [1e3, 1e5]
    from oracle.parallel import propagate_parallel

    probs = wl.batched_instances()
    total_steps = sum(p.n_steps for p in probs)
    sample = batched_sample(probs)
    R_sample = {i: propagate_parallel(probs[i].H0, probs[i].Hk, probs[i].c, probs[i].dt, probs[i].integrator)
                for i in sample}
    forms = {}
    for prec in ("fp32", "fp32_tc_tf32x3", "fp32_tc_bf16x3"):
        inst, keep, outs = prop.batch([(p.H0, p.Hk, p.c, p.dt, p.n_steps) for p in probs], prec)
        leaf, items, tune_ms, cuda_mask = prop.batch_autotune(inst, prec)
        per = time_launches(torch, lambda: prop.propagate_batched(inst, prec), 5, 2, flush)
        ms = statistics.mean(per)
        Us = [U.cpu().numpy().astype(np.complex128) for U in outs]
        forms[prec] = {"steps_per_s": total_steps / (ms * 1e-3), "ms": ms, "cuda_graph": True,
                       "autotuned": {"leaf_steps": leaf, "items_per_sm": items,
                                     "cuda_core_classes": cuda_mask},
                       "product_backends": prop.stats()["product_backends"],
                       "max_abs_err_vs_oracle_sample": max(float(np.max(np.abs(Us[i] - R_sample[i])))
                                                           for i in sample), "U": Us}
        del keep, outs
    # plain FP64 GPU path: one propagate per instance
    U64 = []
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record()
    for p in probs:
        prop.set_hamiltonians(torch.as_tensor(p.H0).to(dev), torch.as_tensor(p.Hk).to(dev), "midpoint")
        prop.set_controls(torch.as_tensor(p.c).to(dev), p.dt, p.n_steps)
        U64.append(prop.propagate("fp64"))
    t1.record()
    torch.cuda.synchronize()
    ms64 = t0.elapsed_time(t1)
    U64 = [U.cpu().numpy() for U in U64]
    err64_sample = max(float(np.max(np.abs(U64[i] - R_sample[i]))) for i in sample)
    for prec, f in forms.items():
        f["max_abs_err_vs_fp64_gpu"] = max(float(np.max(np.abs(a - b))) for a, b in zip(f.pop("U"), U64))
    out["batched_256_instances_d2to64"] = {
        "total_steps": total_steps, "n_instances": len(probs),
        "oracle_sample": f"{len(sample)} instances: the longest of each dimension and 8 drawn with seed 20210816",
        "fp32_batched": forms["fp32"], "fp32_tc_tf32x3_batched": forms["fp32_tc_tf32x3"],
        "fp32_tc_bf16x3_batched": forms["fp32_tc_bf16x3"],
        "fp64_gpu_per_instance_loop": {"steps_per_s": total_steps / (ms64 * 1e-3), "ms": ms64,
                                       "max_abs_err_vs_oracle_sample": err64_sample,
                                       "note": "set_hamiltonians + set_controls + propagate per instance, "
                                               "the set-up synchronises"},
        "speedup_fp32_batched_vs_fp64_loop": ms64 / forms["fp32"]["ms"]}
    del U64

    # ---- dense precision stress: d = 128, GL4, N = 2^16 (FP64 timed on 2^12 slices)
    prob = wl.dense_stress()
    small = wl.dense_stress(n_steps=1 << 12)
    R = propagate_parallel(prob.H0, prob.Hk, prob.c, prob.dt, prob.integrator)
    res = {}
    for name, prb in (("full", prob), ("small", small)):
        for prec in ("fp32", "fp32_tc_tf32x3", "fp32_tc_bf16x3", "fp64"):
            if name == "small" and prec != "fp64":
                continue
            cdt = torch.complex128 if prec == "fp64" else torch.complex64
            rdt = torch.float64 if prec == "fp64" else torch.float32
            prop.set_hamiltonians(torch.as_tensor(prb.H0).to(cdt), torch.as_tensor(prb.Hk).to(cdt), prb.integrator)
            prop.set_controls(torch.as_tensor(prb.c).to(rdt).to(dev), prb.dt, prb.n_steps)
            U = torch.empty(128, 128, dtype=cdt, device=dev)
            if name == "full" and prec == "fp64":  # one launch for the error (about 9 s)
                prop.propagate(prec, out=U)
                torch.cuda.synchronize()
                per = [float("nan")]
            else:
                per = time_launches(torch, lambda: prop.propagate(prec, out=U), 3 if prec != "fp64" else 1, 1, flush)
            st = prop.stats()
            res[(name, prec)] = (statistics.mean(per), U.cpu().numpy().astype(np.complex128), st)
    d128 = {}
    for prec in ("fp32", "fp32_tc_tf32x3", "fp32_tc_bf16x3"):
        ms, U, st = res[("full", prec)]
        fl = flops_per_launch(st)
        d128[prec] = {"steps_per_s": prob.n_steps / (ms * 1e-3), "ms": ms,
                      "algorithmic_tflops": fl / (ms * 1e-3) / 1e12,
                      "product_backends": st["product_backends"],
                      "max_abs_err_vs_oracle": float(np.max(np.abs(U - R)))}
    d128["fp32"]["roofline"] = roofline_alu(d128["fp32"]["algorithmic_tflops"], "fp32")
    # tcgen05 products: the method's 8 d^3 flops per complex product against the pipe's peak, and
    # the tensor pipe's own work (3 TF32 or 6 BF16 MMA flops per real flop) as utilisation
    for prec, fmt, mult in (("fp32_tc_tf32x3", "tf32", 3.0), ("fp32_tc_bf16x3", "bf16", 6.0)):
        ach = d128[prec]["algorithmic_tflops"]
        pk, note = tensor_peak(fmt)
        d128[prec]["roofline"] = {"bound": "tensor", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                                  "frac": ach / pk, "tensor_utilisation": mult * ach / pk,
                                  "kernel": f"large_kernel<float, 128, GL4, tcgen05 {fmt}>", "peak_note": note}
    ms, _, st = res[("small", "fp64")]
    d128["fp64"] = {"steps_per_s": small.n_steps / (ms * 1e-3), "ms_N4096": ms,
                    "algorithmic_tflops": flops_per_launch(st) / (ms * 1e-3) / 1e12,
                    "max_abs_err_vs_oracle": float(np.max(np.abs(res[("full", "fp64")][1] - R)))}
    d128["fp64"]["roofline"] = roofline_alu(d128["fp64"]["algorithmic_tflops"], "fp64")
    d128["speedup_tf32x3_vs_fp64"] = d128["fp32_tc_tf32x3"]["steps_per_s"] / d128["fp64"]["steps_per_s"]
    out["dense_stress_d128_magnus4_gl2_N65536"] = d128
    prop.close()
    return out


def run_ours(args):
    import numpy as np
    import torch

    rank, local, world = dist_setup("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2108_07126_gb300 import binding as b
    from paper_2108_07126_gb300 import workloads as wl

    prob = wl.coupled_spins(n_steps=args.n_steps)
    N = prob.n_steps
    prop = b.Propagator(local)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    # ---- FP32 path (headline)
    H0 = torch.as_tensor(prob.H0).to(torch.complex64)
    Hk = torch.as_tensor(prob.Hk).to(torch.complex64)
    c32 = torch.as_tensor(prob.c).to(torch.float32).to(dev)
    prop.set_hamiltonians(H0, Hk, prob.integrator)
    prop.set_controls(c32, prob.dt, N)
    U32 = torch.empty(16, 16, dtype=torch.complex64, device=dev)
    fn32 = lambda: prop.propagate("fp32", out=U32)

    gpu_uuid = str(torch.cuda.get_device_properties(dev).uuid)
    clocks = ClockSampler(gpu_uuid if gpu_uuid.startswith("GPU-") else f"GPU-{gpu_uuid}")
    barrier(world)
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    per32 = time_launches(torch, fn32, args.steps, args.warmup, flush)
    torch.cuda.synchronize()
    barrier(world)
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    st32 = prop.stats()
    ms32 = max_over_ranks(statistics.mean(per32), world, dev)
    U32h = U32.cpu().numpy().astype(np.complex128)

    # ---- plain FP64 GPU path on the same workload
    prop.set_hamiltonians(torch.as_tensor(prob.H0), torch.as_tensor(prob.Hk), prob.integrator)
    c64 = torch.as_tensor(prob.c).to(dev)
    prop.set_controls(c64, prob.dt, N)
    U64 = torch.empty(16, 16, dtype=torch.complex128, device=dev)
    per64 = time_launches(torch, lambda: prop.propagate("fp64", out=U64), args.fp64_steps, 1, flush)
    st64 = prop.stats()
    ms64 = max_over_ranks(statistics.mean(per64), world, dev)
    U64h = U64.cpu().numpy()
    err32 = float(np.max(np.abs(U32h - U64h)))
    unit_err = float(np.max(np.abs(U64h.conj().T @ U64h - np.eye(16))))
    # both paths against the FP64 oracle on the full workload (exact inputs), rank 0 only
    err32_oracle = err64_oracle = None
    if rank == 0:
        from oracle.parallel import propagate_parallel

        R = propagate_parallel(prob.H0, prob.Hk, prob.c, prob.dt, prob.integrator)
        err32_oracle = float(np.max(np.abs(U32h - R)))
        err64_oracle = float(np.max(np.abs(U64h - R)))

    # ---- end to end through the C ABI with host buffers (pinned controls in, host U out)
    c_host = torch.as_tensor(prob.c).to(torch.float32).pin_memory()
    U_host = np.zeros((16, 16), np.complex64)
    prop.set_hamiltonians(H0, Hk, prob.integrator)
    e2e_times = []
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.parament_set_controls(prop.ctx, c_host.data_ptr(), b.PARAMENT_F32, N, prob.dt)
        b.parament_propagate(prop.ctx, U_host.ctypes.data, b.PARAMENT_PREC_FP32)
        t1 = time.perf_counter()
        if i >= args.warmup:
            e2e_times.append(t1 - t0)
    e2e_s = max_over_ranks(statistics.mean(e2e_times), world, dev)
    prop.close()

    # ---- measured pipe rates for the rooflines (rank 0, outside the timed regions)
    if rank == 0:
        measure_peaks(b, local)

    # ---- secondary workloads (reported beside the headline, not part of `value`)
    extra = {}
    if rank == 0 and not args.no_extra:
        extra = secondary_workloads(torch, b, wl, dev, flush)

    # ---- CPU baseline: the oracle on a bounded sample, rank 0 only
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        o = time_oracle(args.cpu_sample)
        cpu = {"value": o["n"] / o["seconds"], "unit": UNIT, "cores": o["cores"], "kind": "oracle",
               "per_core_value": o["one_core_rate"],
               "sample": f"first {o['n']} slices of the workload, FP64 eigendecomposition oracle, cut into "
                         f"{o['cores']} contiguous ranges, one single-threaded process each"}

    if rank != 0:
        return
    fl32 = flops_per_launch(st32)
    fl64 = flops_per_launch(st64)
    ach32 = fl32 / (statistics.mean(per32) * 1e-3) / 1e12
    ach64 = fl64 / (statistics.mean(per64) * 1e-3) / 1e12
    roof32 = roofline_alu(ach32, "fp32")
    roof64 = roofline_alu(ach64, "fp64")
    value = world * N / (ms32 * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms32, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(workload_config(N, "fp32"), parallelism=("replicas" if world > 1 else "single"),
                       n_basis_kept=st32["n_basis"]),
        "max_abs_err_vs_oracle": err32_oracle,
        "fp64_gpu": {"value": world * N / (ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64,
                     "steps": args.fp64_steps, "max_abs_err_vs_oracle": err64_oracle,
                     "max_abs_err_vs_oracle_bound": 1e-11,
                     "unitarity_err": unit_err, "exp_products": st64["exp_products"],
                     "max_degree": st64["max_degree"], "max_squarings": st64["max_squarings"],
                     "roofline": roof64},
        "speedup_vs_fp64_gpu": ms64 / ms32,
        "max_abs_err_vs_fp64_gpu": err32,
        "kernel": {"grid_blocks": st32["grid_blocks"], "block_threads": st32["block_threads"],
                   "leaves": st32["leaves"], "exp_products": st32["exp_products"],
                   "tree_products": st32["tree_products"], "max_degree": st32["max_degree"],
                   "max_squarings": st32["max_squarings"], "flops_per_launch": fl32},
        "roofline": dict(roof32, traffic=TRAFFIC_BYTES_PER_SLICE * N, traffic_note=TRAFFIC_NOTE),
        "peaks": dict(MEASURED, bf16_cublas_tflops_pool=PEAKS.get("bf16_tflops"),
                      note="measured by parament_measure_peaks in this run, after the timed region"),
        "cpu_baseline": cpu,
        "e2e": {"value": world * N / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(c_host.numel() * 4),
                "d2h_bytes_per_step": int(U_host.nbytes)},
        "secondary": extra,
        "gpu_launches": args.steps,
        "clocks": clk,
        "wall_s_timed": t_wall,
    }
    print(json.dumps(line))


_SCALING_CPU = """
import json, sys, time
sys.path.insert(0, {root!r})
import oracle
from paper_2108_07126_gb300 import workloads as wl
out = []
for d, n in {cases!r}:
    prob = wl.random_problem(d, 2, n, "midpoint", seed=20210816 + d, g_norm=0.3)
    t0 = time.perf_counter()
    U = oracle.propagate(prob.H0, prob.Hk, prob.c, prob.dt, prob.integrator)
    out.append([d, n, time.perf_counter() - t0])
print(json.dumps(out))
"""


def run_scaling(args):
    """The paper's performance experiments (Sec. 5) on this GPU, synthetic dense input.

    E1 (run time vs matrix size, 80 000 time steps): d = 2 .. 192, FP32 and FP64, controls
    resident on the device, CUDA events around parament_propagate.  E3 (run time vs time
    steps for d = 2, 40, 192): end to end through the C ABI from host memory (controls in,
    U out, one call each, host wall clock), FP32 and FP64, against the FP64 oracle on one
    host core; the crossover is where the FP64 GPU call becomes faster than the oracle.
    Input: workloads.random_problem(d, K = 2, N, midpoint, g_norm = 0.3): GUE drift, two GUE
    controls, Gaussian samples.  Runs that would take more than ~10 s are skipped.
    """
    import numpy as np
    import torch

    from paper_2108_07126_gb300 import binding as b
    from paper_2108_07126_gb300 import workloads as wl

    dev = torch.device("cuda", 0)
    prop = b.Propagator(0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > L2, written between timed calls
    results = {"e1": [], "e3_gpu": [], "e3_cpu": []}
    os.makedirs(os.path.dirname(os.path.abspath(args.scaling_out)), exist_ok=True)
    record = open(args.scaling_out, "w")

    def emit(kind, row):
        line = json.dumps({kind: row})
        record.write(line + "\n")
        record.flush()
        print(line, flush=True)

    emit("meta", {"gpu": torch.cuda.get_device_name(dev), "torch": torch.__version__,
                  "input": "random_problem(d, K=2, N, midpoint, g_norm=0.3): GUE drift, two GUE controls, "
                           "Gaussian samples, seed 20210816 + d"})

    def problem(d, n):
        return wl.random_problem(d, 2, n, "midpoint", seed=20210816 + d, g_norm=0.3)

    def load(prob, prec, device_ctrl=True):
        cdt = torch.complex128 if prec == "fp64" else torch.complex64
        prop.set_hamiltonians(torch.as_tensor(prob.H0).to(cdt), torch.as_tensor(prob.Hk).to(cdt), "midpoint")
        if device_ctrl:
            rdt = torch.float64 if prec == "fp64" else torch.float32
            prop.set_controls(torch.as_tensor(prob.c).to(rdt).to(dev), prob.dt, prob.n_steps)
        return cdt

    # ---- E1: run time vs d at 80 000 time steps (every run on the full 80 000 steps; calls of
    #      more than ~5 s are timed once after a short warm-up call)
    n1 = 80000
    dims = (2, 4, 8, 12, 16, 24, 32, 40, 48, 64, 96, 128, 160, 192)
    for prec in ("fp32", "fp64", "fp32_tc_tf32x3"):
        rate = None
        for d in dims:
            if prec == "fp32_tc_tf32x3" and d <= 16:
                continue
            prob = problem(d, n1)
            cdt = load(prob, "fp64" if prec == "fp64" else "fp32")
            U = torch.empty(d, d, dtype=cdt, device=dev)
            if rate is not None and n1 / rate > 5.0:
                prop.propagate(prec, out=U)  # warm-up (kernels loaded, workspace sized)
                torch.cuda.synchronize()
                per = time_launches(torch, lambda: prop.propagate(prec, out=U), 1, 0, flush)
            else:
                per = time_launches(torch, lambda: prop.propagate(prec, out=U), 3, 1, flush)
            ms = statistics.median(per)
            rate = n1 / (ms * 1e-3)
            st = prop.stats()
            row = {"d": d, "padded": pad_dim(d), "prec": prec, "n_steps": n1, "ms": ms,
                   "steps_per_s": rate, "timed_calls": len(per), "product_backends": st["product_backends"],
                   "algorithmic_tflops": flops_per_launch(st) / (ms * 1e-3) / 1e12}
            results["e1"].append(row)
            emit("e1", row)

    # ---- E3: run time vs N, end to end from host memory, against the oracle
    grid = (1, 10, 100, 1000, 10000, 100000, 1000000)
    for d in (2, 40, 192):
        for prec in ("fp32", "fp64"):
            rate = None
            for n in grid:
                if rate is not None and n / rate > 10.0:
                    break
                prob = problem(d, n)
                cdt = load(prob, prec, device_ctrl=False)
                rdt = torch.float64 if prec == "fp64" else torch.float32
                c_host = torch.as_tensor(prob.c).to(rdt).contiguous().pin_memory()
                U_host = np.zeros((d, d), np.complex128 if prec == "fp64" else np.complex64)
                pc = b.PARAMENT_PREC_FP64 if prec == "fp64" else b.PARAMENT_PREC_FP32
                cd = b.PARAMENT_F64 if prec == "fp64" else b.PARAMENT_F32

                def call():
                    b.parament_set_controls(prop.ctx, c_host.data_ptr(), cd, n, prob.dt)
                    b.parament_propagate(prop.ctx, U_host.ctypes.data, pc)  # host U: returns after the copy

                call()
                ts = []
                for _ in range(5 if n <= 10000 else 2):
                    t0 = time.perf_counter()
                    call()
                    ts.append(time.perf_counter() - t0)
                sec = statistics.median(ts)
                rate = n / sec
                row = {"d": d, "prec": prec, "n_steps": n, "seconds": sec}
                results["e3_gpu"].append(row)
                emit("e3_gpu", row)
    prop.close()

    # CPU side: the FP64 oracle on one host core, in a fresh process, within ~10 s per size
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = "1"
    for d, cap in ((2, 100000), (40, 10000), (192, 100)):
        cases = [(d, n) for n in grid if n <= cap]
        code = _SCALING_CPU.format(root=ROOT, cases=cases)
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
        if r.returncode != 0:
            raise RuntimeError(r.stderr)
        for dd, n, sec in json.loads(r.stdout.strip().splitlines()[-1]):
            row = {"d": dd, "n_steps": n, "seconds": sec, "cores": 1}
            results["e3_cpu"].append(row)
            emit("e3_cpu", row)

    # crossover (FP64): first N on the grid where the GPU call beats the oracle, log-log
    # interpolated between the neighbouring grid points
    cross = {}
    for d in (2, 40, 192):
        g = {r["n_steps"]: r["seconds"] for r in results["e3_gpu"] if r["d"] == d and r["prec"] == "fp64"}
        c = {r["n_steps"]: r["seconds"] for r in results["e3_cpu"] if r["d"] == d}
        common = sorted(set(g) & set(c))
        val = None
        for i, n in enumerate(common):
            if g[n] < c[n]:
                if i == 0:
                    val = {"n_steps": n, "note": "GPU faster already at the smallest N"}
                else:
                    n0 = common[i - 1]
                    r0 = math.log(g[n0] / c[n0])
                    r1 = math.log(g[n] / c[n])
                    x = math.log(n0) + (math.log(n) - math.log(n0)) * r0 / (r0 - r1)
                    val = {"n_steps": math.exp(x), "between": [n0, n]}
                break
        cross[d] = val
    emit("scaling_summary", {"crossover_fp64": cross, "input": "random_problem(d, 2, N, midpoint, g_norm=0.3), "
                                                            "GUE drift and controls", "cpu": "FP64 oracle, one core"})
    record.close()


def pad_dim(d: int) -> int:
    """Padded dimension the library runs d at (next power of two, at least 2)."""
    p = 2
    while p < d:
        p *= 2
    return p


def scaling_report(path: str) -> str:
    """Markdown tables (run time vs d; run time vs N with the CPU oracle) of a --scaling record."""
    rows = [json.loads(line) for line in open(path) if line.strip()]
    e1 = [r["e1"] for r in rows if "e1" in r]
    g3 = [r["e3_gpu"] for r in rows if "e3_gpu" in r]
    c3 = [r["e3_cpu"] for r in rows if "e3_cpu" in r]
    summ = [r["scaling_summary"] for r in rows if "scaling_summary" in r]
    out = []
    dims = sorted({r["d"] for r in e1})
    precs = [p for p in ("fp32", "fp32_tc_tf32x3", "fp64") if any(r["prec"] == p for r in e1)]
    out.append("| d (padded) | " + " | ".join(f"{d} ({pad_dim(d)})" if pad_dim(d) != d else str(d) for d in dims) + " |")
    out.append("|---" * (len(dims) + 1) + "|")
    for p in precs:
        cells = []
        for d in dims:
            r = [x for x in e1 if x["d"] == d and x["prec"] == p]
            cells.append(f"{r[0]['ms']:.4g}" if r else "—")
        out.append(f"| {p} ms | " + " | ".join(cells) + " |")
    out.append("")
    ns = sorted({r["n_steps"] for r in g3} | {r["n_steps"] for r in c3})
    ds = sorted({r["d"] for r in g3})
    head = ["N"] + [f"d={d} {p}" for d in ds for p in ("fp32", "fp64", "cpu")]
    out.append("| " + " | ".join(head) + " |")
    out.append("|---" * len(head) + "|")

    def fmt(sec):
        return f"{sec * 1e3:.3g} ms" if sec < 1.0 else f"{sec:.3g} s"

    for n in ns:
        cells = [f"{n:g}"]
        for d in ds:
            for p in ("fp32", "fp64"):
                r = [x for x in g3 if x["d"] == d and x["prec"] == p and x["n_steps"] == n]
                cells.append(fmt(r[0]["seconds"]) if r else "—")
            r = [x for x in c3 if x["d"] == d and x["n_steps"] == n]
            cells.append(fmt(r[0]["seconds"]) if r else "—")
        out.append("| " + " | ".join(cells) + " |")
    if summ:
        out.append("")
        out.append("FP64 crossover (GPU call faster than the one-core oracle): " + json.dumps(summ[-1]["crossover_fp64"]))
    return "\n".join(out)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.scaling_report:
        print(scaling_report(args.scaling_out))
    elif args.scaling:
        run_scaling(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
