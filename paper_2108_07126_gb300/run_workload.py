"""Run one of the synthetic workloads through the library and print its timing as JSON.

    python -m paper_2108_07126_gb300.run_workload --workload spins --prec fp32 --n-steps 262144 --reps 3

Workloads: ``rabi`` (d = 2, midpoint), ``spins`` (d = 16, GL4 Magnus), ``gradient``
(d = 8, loss + adjoint gradient), ``dense`` (d = 128, GL4 Magnus), ``batched``
(mixed instances, d up to 64, one persistent launch), ``random`` (dense random problem of
dimension ``--dim``, two controls, midpoint, ||G|| ~ 0.3).  ``--exp chebyshev`` selects the
paper's Chebyshev exponential, ``--traj-every n`` times the trajectory U(t_n) instead of
U(T).  Times are CUDA events on the
launching stream around each call, after one warm-up call.
"""

from __future__ import annotations

import argparse
import json
import statistics

import torch

from . import binding as b
from . import workloads as wl


def _time(fn, reps):
    fn()
    torch.cuda.synchronize()
    out = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        e.record()
        torch.cuda.synchronize()
        out.append(a.elapsed_time(e))
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", choices=["rabi", "spins", "gradient", "dense", "batched", "random"],
                    default="spins")
    ap.add_argument("--dim", type=int, default=64, help="dimension of the random workload")
    ap.add_argument("--prec", default="fp32")
    ap.add_argument("--n-steps", type=int, default=0, help="slices (0 = the workload's default)")
    ap.add_argument("--n-inst", type=int, default=256, help="instances of the batched workload")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--exp", choices=["taylor", "chebyshev"], default="taylor", help="exponential of propagate")
    ap.add_argument("--traj-every", type=int, default=0,
                    help="time the trajectory U(t_n) every this many slices instead of U(T)")
    args = ap.parse_args(argv)
    prec = args.prec
    cdt = torch.complex128 if prec == "fp64" else torch.complex64
    rdt = torch.float64 if prec == "fp64" else torch.float32
    prop = b.Propagator(0)
    res = {"workload": args.workload, "prec": prec}
    if args.workload == "batched":
        probs = wl.batched_instances(n_inst=args.n_inst)
        inst, keep, outs = prop.batch([(p.H0, p.Hk, p.c, p.dt, p.n_steps) for p in probs], prec)
        ms = _time(lambda: prop.propagate_batched(inst, prec), args.reps)
        res["n_steps"] = sum(p.n_steps for p in probs)
    else:
        make = {"rabi": wl.rabi_qubit, "spins": wl.coupled_spins, "gradient": wl.gradient_qubits,
                "dense": wl.dense_stress,
                "random": lambda n_steps=4096: wl.random_problem(args.dim, 2, n_steps, "midpoint", seed=5,
                                                                 g_norm=0.3)}[args.workload]
        prob = make(n_steps=args.n_steps) if args.n_steps else make()
        if args.exp == "chebyshev":
            prop.set_option(b.PARAMENT_OPT_EXP_METHOD, 1)
        prop.set_hamiltonians(torch.as_tensor(prob.H0).to(cdt), torch.as_tensor(prob.Hk).to(cdt), prob.integrator)
        prop.set_controls(torch.as_tensor(prob.c).to(rdt).cuda(), prob.dt, prob.n_steps)
        res["n_steps"] = prob.n_steps
        if args.workload == "gradient":
            V = torch.as_tensor(prob.V).to(cdt).cuda()
            ms = _time(lambda: prop.propagate_grad(V, prec), args.reps)
        elif args.traj_every > 0:
            n_out = -(-prob.n_steps // args.traj_every)
            T = torch.empty(n_out, prob.dim, prob.dim, dtype=cdt, device="cuda")
            ms = _time(lambda: prop.propagate_trajectory(prec, args.traj_every, out=T), args.reps)
            res["traj_outputs"] = n_out
        else:
            U = torch.empty(prob.dim, prob.dim, dtype=cdt, device="cuda")
            ms = _time(lambda: prop.propagate(prec, out=U), args.reps)
        res["stats"] = prop.stats()
    res["ms"] = ms
    res["steps_per_s"] = res["n_steps"] / (statistics.mean(ms) * 1e-3)
    prop.close()
    print(json.dumps(res))


if __name__ == "__main__":
    main()
