"""The benchmark workloads at their full size against the FP64 oracle (exact inputs).

Every precision is compared with the oracle's U(T) (eigendecomposition exponentials, ordered
product; spread over the host cores by ``oracle.parallel``), in the launch configuration the
benchmark times.  FP64 must stay within 1e-11.  The reduced-precision paths see the inputs rounded
to complex64 / float32, so their error contains that rounding too; each has a bound a few times
its measured error (the bounds and the measurements behind them are listed with the tolerances of
the design notes), tight enough that a regression by a factor of a few fails.
"""

import numpy as np
import pytest

from oracle.parallel import propagate_parallel
from paper_2108_07126_gb300 import workloads as wl
from tolerances import FULL_SIZE, TOL64, check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


@pytest.fixture()
def prop(torch):
    from paper_2108_07126_gb300.binding import Propagator

    p = Propagator(0)
    yield p
    p.close()


def run(prop, prob, prec):
    import torch

    hd = torch.complex128 if prec == "fp64" else torch.complex64
    cd = torch.float64 if prec == "fp64" else torch.float32
    prop.set_hamiltonians(torch.as_tensor(prob.H0).to(hd), torch.as_tensor(prob.Hk).to(hd), prob.integrator)
    prop.set_controls(torch.as_tensor(prob.c).to(cd).cuda(), prob.dt, prob.n_steps)
    U = prop.propagate(prec)
    torch.cuda.synchronize()
    return U.cpu().numpy().astype(np.complex128)


def oracle_u(prob):
    return propagate_parallel(prob.H0, prob.Hk, prob.c, prob.dt, prob.integrator)


def test_coupled_spins_full_size(prop):
    """The headline workload (d = 16, GL4 Magnus, N = 2^20): FP64 within 1e-11 of the oracle, FP32
    within its bound."""
    prob = wl.coupled_spins()
    R = oracle_u(prob)
    check(np.max(np.abs(run(prop, prob, "fp64") - R)), TOL64, "coupled spins fp64")
    check(np.max(np.abs(run(prop, prob, "fp32") - R)), FULL_SIZE["coupled_spins"]["fp32"], "coupled spins fp32")


def test_dense_stress_full_size_vs_oracle(prop):
    """d = 128 dense stress (GL4, N = 2^16, ||G||_1 ~ 3.9: degree and squarings): every precision
    against the oracle."""
    prob = wl.dense_stress()
    R = oracle_u(prob)
    check(np.max(np.abs(run(prop, prob, "fp64") - R)), TOL64, "dense fp64")
    for prec in ("fp32", "fp32_tc_tf32x3", "fp32_tc_bf16x3"):
        check(np.max(np.abs(run(prop, prob, prec) - R)), FULL_SIZE["dense_stress"][prec], ("dense", prec))


def batched_sample(probs):
    """The longest instance of every dimension and eight instances drawn with a fixed seed."""
    picked = set()
    for d in sorted({p.dim for p in probs}):
        picked.add(max((i for i, p in enumerate(probs) if p.dim == d), key=lambda i: probs[i].n_steps))
    rng = np.random.default_rng(20210816)
    picked.update(int(i) for i in rng.choice(len(probs), 8, replace=False))
    return sorted(picked)


@pytest.mark.parametrize("prec", ["fp32", "fp32_tc_tf32x3", "fp32_tc_bf16x3"])
def test_batched_sweep_sample_vs_oracle(prop, prec):
    """All 256 instances of the batched sweep in one autotuned launch; a sample of them (the
    longest of each dimension and eight more) against the oracle."""
    import torch

    probs = wl.batched_instances()
    inst, keep, outs = prop.batch([(p.H0, p.Hk, p.c, p.dt, p.n_steps) for p in probs], prec)
    prop.batch_autotune(inst, prec)
    prop.propagate_batched(inst, prec)
    torch.cuda.synchronize()
    for i in batched_sample(probs):
        p = probs[i]
        err = np.max(np.abs(outs[i].cpu().numpy().astype(np.complex128) - oracle_u(p)))
        check(err, FULL_SIZE["batched"][prec], ("batched", prec, p.name))
