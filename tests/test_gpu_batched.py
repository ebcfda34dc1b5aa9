"""Batched propagation of instances with uneven dimension and step count (one persistent launch)."""

import numpy as np
import pytest

import oracle
from paper_2108_07126_gb300 import workloads as wl
from tolerances import TOL64, U32, check, tol32, tol_tc  # noqa: F401

pytestmark = pytest.mark.gpu



@pytest.fixture()
def prop():
    import torch

    from paper_2108_07126_gb300.binding import Propagator

    assert torch.cuda.is_available()
    p = Propagator(0)
    yield p
    p.close()


def mixed_batch(integrator="midpoint", seed=0):
    rng = np.random.default_rng(seed)
    shapes = [(2, 1, 0), (2, 2, 1), (3, 2, 777), (4, 3, 5000), (8, 2, 3001), (16, 4, 20000), (5, 1, 129),
              (32, 2, 600), (64, 3, 300), (12, 2, 2048), (40, 2, 97), (16, 6, 1)]
    probs = []
    for i, (d, K, n) in enumerate(shapes):
        probs.append(wl.random_problem(d, K, n, integrator, seed=int(rng.integers(1 << 30)), g_norm=0.3))
    return probs


def refs(probs, rounded=False):
    out = []
    for p in probs:
        if rounded:
            out.append(oracle.propagate(p.H0.astype(np.complex64).astype(np.complex128),
                                        p.Hk.astype(np.complex64).astype(np.complex128),
                                        p.c.astype(np.float32).astype(np.float64), p.dt, p.integrator))
        else:
            out.append(oracle.propagate(p.H0, p.Hk, p.c, p.dt, p.integrator))
    return out


@pytest.mark.parametrize("graph", [1, 0])
@pytest.mark.parametrize("integrator", ["midpoint", "magnus4_gl2"])
def test_batched_fp64_matches_oracle(prop, graph, integrator):
    import torch

    from paper_2108_07126_gb300 import binding as b

    probs = mixed_batch(integrator, seed=1)
    prop.set_option(b.PARAMENT_OPT_BATCH_GRAPH, graph)
    inst, keep, outs = prop.batch([(p.H0, p.Hk, p.c, p.dt, p.n_steps) for p in probs], "fp64")
    R = refs(probs)
    for rep in range(2):  # the second call replays the captured graph
        for U in outs:
            U.fill_(float("nan"))
        prop.propagate_batched(inst, "fp64", integrator)
        torch.cuda.synchronize()
        for p, U, r in zip(probs, outs, R):
            assert np.max(np.abs(U.cpu().numpy() - r)) <= TOL64, (p.name, rep)


@pytest.mark.parametrize("integrator", ["midpoint", "magnus4_gl2"])
@pytest.mark.parametrize("prec", ["fp32", "fp32_tc_tf32x3", "fp32_tc_bf16x3"])
def test_batched_fp32_matches_oracle(prop, prec, integrator):
    import torch

    from paper_2108_07126_gb300 import binding as b

    probs = mixed_batch(integrator, seed=2) + [wl.random_problem(100, 2, 33, integrator, seed=77, g_norm=0.3),
                                               wl.random_problem(128, 1, 20, integrator, seed=78, g_norm=0.3)]
    inst, keep, outs = prop.batch([(p.H0, p.Hk, p.c, p.dt, p.n_steps) for p in probs], prec)
    prop.propagate_batched(inst, prec, integrator)
    torch.cuda.synchronize()
    for p, U, r in zip(probs, outs, refs(probs, rounded=True)):
        err = np.max(np.abs(U.cpu().numpy().astype(np.complex128) - r))
        check(err, (tol32 if prec == "fp32" else tol_tc)(p.dim, p.n_steps), (p.name, err))
    st = prop.stats()
    want = b.PARAMENT_BACKEND_CUDA_CORES | (0 if prec == "fp32" else b.PARAMENT_BACKEND_TCGEN05)
    assert st["product_backends"] == want and st["device_status"] == 0


@pytest.mark.parametrize("prec", ["fp32_tc_tf32x3", "fp32_tc_bf16x3"])
def test_batched_tensor_core_classes_on_cuda_cores(prop, prec):
    """PARAMENT_OPT_BATCH_CUDA_CORE_CLASSES moves chosen dimension classes back to the CUDA cores;
    the autotuner picks a mask and reports it."""
    import torch

    from paper_2108_07126_gb300 import binding as b

    probs = mixed_batch("midpoint", seed=4) + [wl.random_problem(128, 1, 20, "midpoint", seed=79, g_norm=0.3)]
    inst, keep, outs = prop.batch([(p.H0, p.Hk, p.c, p.dt, p.n_steps) for p in probs], prec)
    R = refs(probs, rounded=True)
    for mask, want in ((0b111, b.PARAMENT_BACKEND_CUDA_CORES),
                       (0b011, b.PARAMENT_BACKEND_CUDA_CORES | b.PARAMENT_BACKEND_TCGEN05)):
        prop.set_option(b.PARAMENT_OPT_BATCH_CUDA_CORE_CLASSES, mask)
        prop.propagate_batched(inst, prec)
        torch.cuda.synchronize()
        assert prop.stats()["product_backends"] == want, mask
        for p, U, r in zip(probs, outs, R):
            err = np.max(np.abs(U.cpu().numpy().astype(np.complex128) - r))
            check(err, tol_tc(p.dim, p.n_steps), (mask, p.name, err))
    leaf, items, ms, mask = prop.batch_autotune(inst, prec)
    assert 0 <= mask <= 7 and ms > 0
    assert prop.get_option(b.PARAMENT_OPT_BATCH_CUDA_CORE_CLASSES) == mask


def test_batched_matches_single_calls(prop):
    """Same inputs through the batched and the per-instance entry points (FP64)."""
    import torch

    probs = mixed_batch("midpoint", seed=3)[:8]
    inst, keep, outs = prop.batch([(p.H0, p.Hk, p.c, p.dt, p.n_steps) for p in probs], "fp64")
    prop.propagate_batched(inst, "fp64")
    torch.cuda.synchronize()
    for p, U in zip(probs, outs):
        prop.set_hamiltonians(torch.as_tensor(p.H0), torch.as_tensor(p.Hk), p.integrator)
        prop.set_controls(torch.as_tensor(p.c), p.dt, p.n_steps)
        Us = prop.propagate("fp64")
        assert torch.max(torch.abs(Us - U)).item() <= 1e-12


def test_batched_workload_sample_and_autotune(prop):
    import torch

    probs = wl.batched_instances(n_inst=24, n_max=2e4)
    inst, keep, outs = prop.batch([(p.H0, p.Hk, p.c, p.dt, p.n_steps) for p in probs], "fp32")
    leaf, items, ms, _ = prop.batch_autotune(inst, "fp32")
    assert leaf in (32, 128) and items in (8, 16, 32, 64) and ms > 0
    prop.propagate_batched(inst, "fp32")
    torch.cuda.synchronize()
    for p, U, r in zip(probs, outs, refs(probs, rounded=True)):
        err = np.max(np.abs(U.cpu().numpy().astype(np.complex128) - r))
        check(err, tol32(p.dim, p.n_steps), (p.name, err))


def test_batched_workload_full_size(prop):
    """All 256 instances of the batched sweep in the benchmark's configuration (autotuned, one FP32
    launch, graph): every U(T) is unitary within the FP32 bound of its instance, and the two
    shortest instances of each dimension match the oracle."""
    import torch

    probs = wl.batched_instances()
    inst, keep, outs = prop.batch([(p.H0, p.Hk, p.c, p.dt, p.n_steps) for p in probs], "fp32")
    prop.batch_autotune(inst, "fp32")
    prop.propagate_batched(inst, "fp32")
    torch.cuda.synchronize()
    Us = [U.cpu().numpy().astype(np.complex128) for U in outs]
    for p, U in zip(probs, Us):
        unit = np.max(np.abs(U.conj().T @ U - np.eye(p.dim)))
        check(unit, tol32(p.dim, p.n_steps), (p.name, unit))
    picked = []
    for d in sorted({p.dim for p in probs}):
        same = sorted((i for i, p in enumerate(probs) if p.dim == d), key=lambda i: probs[i].n_steps)
        picked += same[:2]
    for i, r in zip(picked, refs([probs[i] for i in picked], rounded=True)):
        err = np.max(np.abs(Us[i] - r))
        check(err, tol32(probs[i].dim, probs[i].n_steps), (probs[i].name, err))


def test_batched_rejects_host_pointers(prop):
    from paper_2108_07126_gb300 import binding as b

    H = np.eye(2, dtype=np.complex64)
    U = np.zeros((2, 2), np.complex64)
    inst = [b.parament_instance(2, 0, H.ctypes.data, None, None, 4, 0.1, U.ctypes.data)]
    with pytest.raises(b.ParamentError) as e:
        b.parament_propagate_batched(prop.ctx, inst, b.PARAMENT_C64, b.PARAMENT_F32, b.PARAMENT_MIDPOINT,
                                     b.PARAMENT_PREC_FP32)
    assert e.value.status == b.PARAMENT_ERR_INVALID_VALUE
