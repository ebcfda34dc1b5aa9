"""Trajectories U(t_n) and states psi(t_n) of the CUDA path against the FP64 oracle.

The oracle multiplies the exact slice propagators sequentially and keeps the
running product at the output slices (n = every, 2 every, ..., N).  The CUDA
path runs the forward tree once, scans the leaf products into exclusive FP64
prefixes and walks every leaf again from its prefix.  Tolerances as for U(T):
FP64 1e-11 max-entry; FP32 tol32 = 24 u sqrt(n) + 16 u (tests/tolerances.py) against the oracle on the
float32-rounded inputs.
"""

import numpy as np
import pytest

import oracle
from paper_2108_07126_gb300 import workloads as wl
from tolerances import TOL64, U32, check, tol32  # noqa: F401

pytestmark = pytest.mark.gpu

INTEGRATORS = ("midpoint", "magnus4_gl2", "magnus4_simpson")


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


def load(prop, prob, prec):
    import torch

    hd = torch.complex128 if prec == "fp64" else torch.complex64
    cd = torch.float64 if prec == "fp64" else torch.float32
    prop.set_hamiltonians(torch.as_tensor(prob.H0).to(hd), torch.as_tensor(prob.Hk).to(hd), prob.integrator)
    prop.set_controls(torch.as_tensor(prob.c).to(cd), prob.dt, prob.n_steps)


def rounded(prob):
    return (prob.H0.astype(np.complex64).astype(np.complex128), prob.Hk.astype(np.complex64).astype(np.complex128),
            prob.c.astype(np.float32).astype(np.float64))


@pytest.mark.parametrize("integrator", INTEGRATORS)
@pytest.mark.parametrize("d", [1, 2, 3, 4, 8, 12, 16])
@pytest.mark.parametrize("n,every", [(1, 1), (37, 1), (101, 7), (1000, 64), (1000, 1000), (50, 200)])
def test_fp64_trajectory_matches_oracle(prop, integrator, d, n, every):
    prob = wl.random_problem(d, 3, n, integrator, seed=2000 + d + n, g_norm=0.4)
    load(prop, prob, "fp64")
    T = prop.propagate_trajectory("fp64", every).cpu().numpy()
    R = oracle.trajectory(prob.H0, prob.Hk, prob.c, prob.dt, integrator, every)
    assert T.shape == R.shape == (len(oracle.trajectory_times(n, every)), d, d)
    assert np.max(np.abs(T - R)) <= TOL64


@pytest.mark.parametrize("integrator", INTEGRATORS)
@pytest.mark.parametrize("d", [2, 4, 8, 16])
def test_fp32_trajectory_matches_oracle(prop, integrator, d):
    n, every = 1000, 9
    prob = wl.random_problem(d, 3, n, integrator, seed=2100 + d, g_norm=0.4)
    load(prop, prob, "fp32")
    T = prop.propagate_trajectory("fp32", every).cpu().numpy().astype(np.complex128)
    H0, Hk, c = rounded(prob)
    R = oracle.trajectory(H0, Hk, c, prob.dt, integrator, every)
    check(np.max(np.abs(T - R)), tol32(d, n))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("d", [2, 5, 16])
def test_state_trajectory_matches_oracle(prop, torch, prec, d):
    n, every = 777, 5
    prob = wl.random_problem(d, 2, n, "magnus4_gl2", seed=2200 + d, g_norm=0.5)
    psi0 = wl.haar_unitary(np.random.default_rng(2201 + d), d)[:, 0]
    load(prop, prob, prec)
    P = prop.propagate_trajectory(prec, every, psi0=psi0).cpu().numpy().astype(np.complex128)
    if prec == "fp64":
        R = oracle.trajectory(prob.H0, prob.Hk, prob.c, prob.dt, prob.integrator, every, psi0=psi0)
        tol = TOL64
    else:
        H0, Hk, c = rounded(prob)
        R = oracle.trajectory(H0, Hk, c, prob.dt, prob.integrator, every,
                              psi0=psi0.astype(np.complex64).astype(np.complex128))
        tol = tol32(d, n)
    assert P.shape == R.shape == (len(oracle.trajectory_times(n, every)), d)
    check(np.max(np.abs(P - R)), tol, prec)


def test_rabi_population_over_time(prop):
    """Resonant circular drive: P_1(t_n) = sin^2(w1 t_n / 2) on the GPU at every output time."""
    w1, t, N, every = 0.1, 40.0, 4000, 100
    prob = wl.circular_drive(N, "magnus4_gl2", 1.0, w1, 1.0, t)
    load(prop, prob, "fp64")
    P = prop.propagate_trajectory("fp64", every, psi0=np.array([1.0, 0.0])).cpu().numpy()
    times = oracle.trajectory_times(N, every) * prob.dt
    assert np.max(np.abs(np.abs(P[:, 1]) ** 2 - np.sin(0.5 * w1 * times) ** 2)) < 1e-10


def test_last_output_is_the_propagator(prop):
    prob = wl.random_problem(8, 3, 5000, "magnus4_gl2", seed=2300, g_norm=0.5)
    for prec, tol in (("fp64", 1e-12), ("fp32", tol32(8, 5000))):
        load(prop, prob, prec)
        T = prop.propagate_trajectory(prec, 1000).cpu().numpy()
        U = prop.propagate(prec).cpu().numpy()
        assert np.max(np.abs(T[-1] - U)) <= tol


@pytest.mark.parametrize("grid,warps", [(1, 1), (3, 2), (7, 8), (0, 0)])
def test_trajectory_independent_of_tree_shape(prop, grid, warps):
    """Leaf boundaries fall anywhere relative to the output slices."""
    from paper_2108_07126_gb300 import binding as b

    prob = wl.random_problem(4, 2, 555, "midpoint", seed=2400, g_norm=0.6)
    R = oracle.trajectory(prob.H0, prob.Hk, prob.c, prob.dt, prob.integrator, 11)
    prop.set_option(b.PARAMENT_OPT_GRID_BLOCKS, grid)
    prop.set_option(b.PARAMENT_OPT_BLOCK_WARPS, warps)
    load(prop, prob, "fp64")
    T = prop.propagate_trajectory("fp64", 11).cpu().numpy()
    assert np.max(np.abs(T - R)) <= TOL64
    assert prop.stats()["grid_blocks"] == (grid or prop.stats()["grid_blocks"])


def test_host_buffers(torch):
    """Host psi0 and host outputs through the raw C entry points."""
    from paper_2108_07126_gb300 import binding as b

    prob = wl.random_problem(3, 2, 90, "magnus4_simpson", seed=2500, g_norm=0.3)
    ctx = b.parament_create(0, None)
    try:
        H0 = np.ascontiguousarray(prob.H0)
        Hk = np.ascontiguousarray(prob.Hk)
        c = np.ascontiguousarray(prob.c)
        b.parament_set_hamiltonians(ctx, 3, 2, H0.ctypes.data, Hk.ctypes.data, b.PARAMENT_C128,
                                    b.PARAMENT_MAGNUS4_SIMPSON)
        b.parament_set_controls(ctx, c.ctypes.data, b.PARAMENT_F64, 90, prob.dt)
        U = np.zeros((9, 3, 3), np.complex128)
        b.parament_propagate_trajectory(ctx, None, U.ctypes.data, 10, b.PARAMENT_PREC_FP64)
        R = oracle.trajectory(prob.H0, prob.Hk, prob.c, prob.dt, prob.integrator, 10)
        assert np.max(np.abs(U - R)) <= TOL64
        psi0 = np.ascontiguousarray(np.array([0.6, 0.8j, 0.0], np.complex128))
        P = np.zeros((9, 3), np.complex128)
        b.parament_propagate_trajectory(ctx, psi0.ctypes.data, P.ctypes.data, 10, b.PARAMENT_PREC_FP64)
        assert np.max(np.abs(P - R @ psi0)) <= TOL64
    finally:
        b.parament_destroy(ctx)


def test_errors_and_empty_run(prop, torch):
    from paper_2108_07126_gb300 import binding as b

    ctx = b.parament_create(0, None)
    try:
        out = torch.zeros(4, 2, 2, dtype=torch.complex128, device="cuda")
        assert b.raw_call("parament_propagate_trajectory", ctx, None, out.data_ptr(), 1, 0) == b.PARAMENT_ERR_STATE
        Hok = torch.eye(2, dtype=torch.complex128, device="cuda")
        assert b.raw_call("parament_set_hamiltonians", ctx, 2, 0, Hok.data_ptr(), None, 1, 0) == b.PARAMENT_OK
        assert b.raw_call("parament_set_controls", ctx, None, 1, 4, 0.5) == b.PARAMENT_OK
        assert b.raw_call("parament_propagate_trajectory", ctx, None, out.data_ptr(), 0, 0) == \
            b.PARAMENT_ERR_INVALID_VALUE
        assert b.raw_call("parament_propagate_trajectory", ctx, None, None, 1, 0) == b.PARAMENT_ERR_INVALID_VALUE
        assert b.raw_call("parament_propagate_trajectory", ctx, None, out.data_ptr(), 1, 3) == \
            b.PARAMENT_ERR_UNSUPPORTED
        assert b.raw_call("parament_propagate_trajectory", ctx, None, out.data_ptr(), 1, 0) == b.PARAMENT_OK
        torch.cuda.synchronize()
        for n in range(4):  # H = I: U(t_n) = exp(-i (n + 1) dt) I
            ref_u = np.eye(2) * np.exp(-1j * 0.5 * (n + 1))
            assert np.max(np.abs(out[n].cpu().numpy() - ref_u)) <= TOL64
        assert b.raw_call("parament_set_option", ctx, b.PARAMENT_OPT_EXP_METHOD, 1) == b.PARAMENT_OK
        assert b.raw_call("parament_propagate_trajectory", ctx, None, out.data_ptr(), 1, 0) == \
            b.PARAMENT_ERR_UNSUPPORTED
        assert b.raw_call("parament_set_option", ctx, b.PARAMENT_OPT_EXP_METHOD, 0) == b.PARAMENT_OK
        assert b.raw_call("parament_set_controls", ctx, None, 1, 0, 0.5) == b.PARAMENT_OK
        assert b.raw_call("parament_propagate_trajectory", ctx, None, None, 3, 0) == b.PARAMENT_OK  # N = 0
        H32 = torch.eye(32, dtype=torch.complex128, device="cuda")
        assert b.raw_call("parament_set_hamiltonians", ctx, 32, 0, H32.data_ptr(), None, 1, 0) == b.PARAMENT_OK
        assert b.raw_call("parament_set_controls", ctx, None, 1, 4, 0.5) == b.PARAMENT_OK
        big = torch.zeros(4, 32, 32, dtype=torch.complex128, device="cuda")
        assert b.raw_call("parament_propagate_trajectory", ctx, None, big.data_ptr(), 1, 3) == \
            b.PARAMENT_ERR_UNSUPPORTED  # tensor-core precision
        assert b.raw_call("parament_propagate_trajectory", ctx, None, big.data_ptr(), 1, 0) == b.PARAMENT_OK
        torch.cuda.synchronize()
        for n in range(4):  # H = I at d = 32 (block-level kernel)
            assert np.max(np.abs(big[n].cpu().numpy() - np.eye(32) * np.exp(-1j * 0.5 * (n + 1)))) <= TOL64
    finally:
        b.parament_destroy(ctx)


@pytest.mark.parametrize("integrator", INTEGRATORS)
@pytest.mark.parametrize("d,n,every", [(20, 37, 5), (40, 100, 7), (64, 33, 33), (128, 9, 2), (192, 5, 3)])
def test_large_d_fp64_trajectory_matches_oracle(prop, integrator, d, n, every):
    """d > 16: one leaf per thread block, FP64 prefixes by a scan over the leaf products."""
    prob = wl.random_problem(d, 2, n, integrator, seed=2600 + d + n, g_norm=0.5)
    load(prop, prob, "fp64")
    T = prop.propagate_trajectory("fp64", every).cpu().numpy()
    R = oracle.trajectory(prob.H0, prob.Hk, prob.c, prob.dt, integrator, every)
    assert T.shape == R.shape
    assert np.max(np.abs(T - R)) <= TOL64


@pytest.mark.parametrize("d", [32, 64, 128])
def test_large_d_fp32_trajectory_and_states(prop, d):
    n, every = (301, 10) if d <= 64 else (41, 4)
    prob = wl.random_problem(d, 2, n, "magnus4_gl2", seed=2700 + d, g_norm=0.4)
    psi0 = wl.haar_unitary(np.random.default_rng(2701 + d), d)[:, 0]
    load(prop, prob, "fp32")
    T = prop.propagate_trajectory("fp32", every).cpu().numpy().astype(np.complex128)
    P = prop.propagate_trajectory("fp32", every, psi0=psi0).cpu().numpy().astype(np.complex128)
    H0, Hk, c = rounded(prob)
    R = oracle.trajectory(H0, Hk, c, prob.dt, prob.integrator, every)
    check(np.max(np.abs(T - R)), tol32(d, n))
    check(np.max(np.abs(P - R @ psi0.astype(np.complex64).astype(np.complex128))), tol32(d, n))
    U = prop.propagate("fp32").cpu().numpy().astype(np.complex128)
    check(np.max(np.abs(T[-1] - U)), 2 * tol32(d, n))


@pytest.mark.parametrize("grid", [1, 3, 152])
def test_large_d_trajectory_independent_of_leaf_count(prop, grid):
    from paper_2108_07126_gb300 import binding as b

    prob = wl.random_problem(48, 2, 160, "midpoint", seed=2800, g_norm=0.5)
    R = oracle.trajectory(prob.H0, prob.Hk, prob.c, prob.dt, prob.integrator, 9)
    prop.set_option(b.PARAMENT_OPT_GRID_BLOCKS, grid)
    load(prop, prob, "fp64")
    T = prop.propagate_trajectory("fp64", 9).cpu().numpy()
    assert np.max(np.abs(T - R)) <= TOL64


def test_coupled_spins_trajectory_slice_of_run(prop):
    """Four coupled spins, GL4, first 2^15 slices of the workload, 32 output times."""
    prob = wl.coupled_spins(n_steps=1 << 15)
    load(prop, prob, "fp64")
    T = prop.propagate_trajectory("fp64", 1024).cpu().numpy()
    R = oracle.trajectory(prob.H0, prob.Hk, prob.c, prob.dt, prob.integrator, 1024)
    assert np.max(np.abs(T - R)) <= 1e-10


def test_coupled_spins_full_size_properties(prop, torch):
    """2^20 slices in the benchmark's launch configuration, 16 output times: every output stays
    unitary and the last one equals U(T) from the propagator within the FP32 bound (twice tol32);
    the first output (2^16 slices) matches the oracle on the same slices."""
    prob = wl.coupled_spins()
    N = prob.n_steps
    load(prop, prob, "fp32")
    T = prop.propagate_trajectory("fp32", 1 << 16).cpu().numpy().astype(np.complex128)
    assert T.shape == (16, 16, 16)
    I = np.eye(16)
    unit = max(np.max(np.abs(U.conj().T @ U - I)) for U in T)
    U = prop.propagate("fp32").cpu().numpy().astype(np.complex128)
    last = np.max(np.abs(T[-1] - U))
    print(f"unitarity {unit:.3e}  last-vs-U(T) {last:.3e}  bound {tol32(16, N):.3e}")
    check(unit, tol32(16, N), unit)
    check(last, 2 * tol32(16, N), last)
    first = wl.coupled_spins(n_steps=1 << 16)
    H0, Hk, c = rounded(first)
    R1 = oracle.propagate(H0, Hk, c, first.dt, first.integrator)
    check(np.max(np.abs(T[0] - R1)), tol32(16, 1 << 16))
