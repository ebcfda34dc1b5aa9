"""Parity of the CUDA propagator with the FP64 oracle, through the C ABI.

Tolerances (tests/tolerances.py).  FP64 path: max-entry |U - U_oracle| <= 1e-11.  FP32
path, against the oracle on the float32-rounded inputs: each slice adds a few units of
u = 2^-24 of rounding per entry (assembly, Taylor polynomial, squarings, leaf product) and the
N slice errors add like a random walk, so the bound is 24 u sqrt(N) + 16 u; the tensor-core
forms get twice that.
"""

import numpy as np
import pytest

import oracle
from paper_2108_07126_gb300 import workloads as wl
from tolerances import FULL_SIZE, TOL64, U32, UNITARY_STEP_2_18, check, tol32, tol_tc  # noqa: F401

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


def run(prop, prob, prec="fp64", c_dtype=None, h_dtype=None):
    import torch

    hd = h_dtype or (torch.complex128 if prec == "fp64" else torch.complex64)
    cd = c_dtype or (torch.float64 if prec == "fp64" else torch.float32)
    prop.set_hamiltonians(torch.as_tensor(prob.H0).to(hd), torch.as_tensor(prob.Hk).to(hd), prob.integrator)
    prop.set_controls(torch.as_tensor(prob.c).to(cd), prob.dt, prob.n_steps)
    U = prop.propagate(prec)
    torch.cuda.synchronize()
    return U.cpu().numpy().astype(np.complex128)


def ref(prob):
    return oracle.propagate(prob.H0, prob.Hk, prob.c, prob.dt, prob.integrator)


def ref32(prob):
    """Oracle on the float32-rounded inputs the FP32 path sees."""
    return oracle.propagate(prob.H0.astype(np.complex64).astype(np.complex128),
                            prob.Hk.astype(np.complex64).astype(np.complex128),
                            prob.c.astype(np.float32).astype(np.float64), prob.dt, prob.integrator)


INTEGRATORS = ("midpoint", "magnus4_gl2", "magnus4_simpson")


@pytest.mark.parametrize("integrator", INTEGRATORS)
@pytest.mark.parametrize("d", [1, 2, 3, 4, 6, 8, 12, 16])
@pytest.mark.parametrize("n", [1, 37, 1000])
def test_fp64_matches_oracle(prop, integrator, d, n):
    prob = wl.random_problem(d, 3, n, integrator, seed=100 + d + n, g_norm=0.4)
    U = run(prop, prob, "fp64")
    assert np.max(np.abs(U - ref(prob))) <= TOL64


@pytest.mark.parametrize("integrator", INTEGRATORS)
@pytest.mark.parametrize("d", [2, 3, 4, 8, 16])
@pytest.mark.parametrize("n", [1, 37, 1000])
def test_fp32_matches_oracle(prop, integrator, d, n):
    prob = wl.random_problem(d, 3, n, integrator, seed=200 + d + n, g_norm=0.4)
    U = run(prop, prob, "fp32")
    check(np.max(np.abs(U - ref32(prob))), tol32(d, n))


@pytest.mark.parametrize("g_norm", [1e-4, 0.05, 0.6, 2.5, 9.0, 40.0])
@pytest.mark.parametrize("d", [2, 8, 16])
def test_norm_range_uses_degree_and_squaring(prop, d, g_norm):
    """Large exponents take squarings, tiny ones low degrees; both stay at FP64 accuracy."""
    prob = wl.random_problem(d, 2, 19, "midpoint", seed=300 + d, g_norm=g_norm)
    U = run(prop, prob, "fp64")
    assert np.max(np.abs(U - ref(prob))) <= TOL64 * max(1.0, g_norm)
    st = prop.stats()
    assert st["tree_products"] == 19
    if g_norm >= 9.0:
        assert st["max_squarings"] >= 3
    assert st["device_status"] == 0


@pytest.mark.parametrize("integrator", ["midpoint", "magnus4_gl2"])
@pytest.mark.parametrize("g_norm", [1e-4, 0.05, 0.6, 2.5, 9.0, 40.0])
def test_fp32_d16_norm_range(prop, integrator, g_norm):
    """FP32 d = 16 (packed two-wide FMA products) through every Paterson-Stockmeyer shape:
    tiny exponents take degree 1 or 2 (no power or one power of X), large ones squarings, whose
    rounding grows with the norm."""
    prob = wl.random_problem(16, 2, 19, integrator, seed=320 + int(10 * g_norm), g_norm=g_norm)
    U = run(prop, prob, "fp32")
    check(np.max(np.abs(U - ref32(prob))), tol32(16, 19) * max(1.0, g_norm))
    st = prop.stats()
    assert st["tree_products"] == 19 and st["device_status"] == 0
    if g_norm <= 1e-4:
        assert st["max_degree"] <= 2
    if g_norm >= 9.0:
        assert st["max_squarings"] >= 2


def test_empty_run_is_identity(prop):
    prob = wl.random_problem(5, 2, 0, "magnus4_gl2", seed=1)
    for prec in ("fp64", "fp32"):
        U = run(prop, prob, prec)
        assert np.array_equal(U, np.eye(5))


def test_zero_basis_matrices_are_dropped(prop):
    """Controls on different qubits commute: their commutator basis matrices are zero and skipped."""
    d = 8
    Hk = np.stack([wl.embed(wl.SX, i, 3) for i in range(3)] + [wl.embed(wl.SY, 0, 3)])
    rng = np.random.default_rng(17)
    H0 = sum(rng.uniform(0.5, 1.5) * wl.embed(wl.SZ, i, 3) for i in range(3))
    c = rng.standard_normal((4, 2 * 300))
    prob = wl.Problem("commuting", H0, Hk, c, 0.05, "magnus4_gl2", 300)
    U = run(prop, prob, "fp64")
    assert np.max(np.abs(U - ref(prob))) <= TOL64
    # 1 + 4 + 4 + 6 coefficients; the sx_i commute with each other and sy_0 commutes with sx_1, sx_2
    assert prop.stats()["n_basis"] == 1 + 4 + 4 + 1


def test_all_zero_hamiltonian(prop):
    prob = wl.Problem("zero", np.zeros((3, 3), np.complex128), np.zeros((2, 3, 3), np.complex128),
                      np.ones((2, 9)), 0.1, "magnus4_simpson", 4)
    for prec in ("fp64", "fp32"):
        assert np.array_equal(run(prop, prob, prec), np.eye(3))


def test_drift_only_is_exact_exponential(prop):
    import scipy.linalg

    rng = np.random.default_rng(7)
    H0 = wl.random_hermitian(rng, 6)
    prob = wl.Problem("drift", H0, np.zeros((0, 6, 6), np.complex128), np.zeros((0, 300)), 0.01, "midpoint", 300)
    U = run(prop, prob, "fp64")
    assert np.max(np.abs(U - scipy.linalg.expm(-1j * H0 * 3.0))) <= TOL64


@pytest.mark.parametrize("grid", [1, 2, 3, 5, 7, 64, 152])
@pytest.mark.parametrize("warps", [1, 3, 8])
def test_tree_shapes_agree(prop, grid, warps):
    """Any split of the slices over blocks, warps and leaves gives the same product."""
    from paper_2108_07126_gb300 import binding as b

    prob = wl.random_problem(4, 2, 4099, "magnus4_gl2", seed=11, g_norm=0.2)
    prop.set_option(b.PARAMENT_OPT_GRID_BLOCKS, grid)
    prop.set_option(b.PARAMENT_OPT_BLOCK_WARPS, warps)
    U = run(prop, prob, "fp64")
    assert np.max(np.abs(U - ref(prob))) <= TOL64
    st = prop.stats()
    assert st["grid_blocks"] == grid and st["block_threads"] == 32 * warps
    assert st["tree_products"] == 4099


def test_deterministic(prop):
    prob = wl.random_problem(16, 4, 3001, "magnus4_gl2", seed=12, g_norm=0.3)
    a = run(prop, prob, "fp32")
    b = run(prop, prob, "fp32")
    assert np.array_equal(a, b)


@pytest.mark.parametrize("m,g_norm", [(1, 1e-9), (2, 1e-6), (4, 0.05), (6, 0.5), (9, 0.5), (12, 0.5)])
def test_forced_taylor_degree(prop, m, g_norm):
    """Forced degrees; low degrees only on small exponents (s squarings amplify rounding by 2^s)."""
    from paper_2108_07126_gb300 import binding as b

    prob = wl.random_problem(8, 2, 50, "midpoint", seed=13, g_norm=g_norm)
    prop.set_option(b.PARAMENT_OPT_TAYLOR_DEGREE, m)
    U = run(prop, prob, "fp64")
    assert np.max(np.abs(U - ref(prob))) <= TOL64
    assert prop.stats()["max_degree"] == m


def test_host_pointers(torch):
    """Host arrays in, host U out, through the raw C entry points."""
    from paper_2108_07126_gb300 import binding as b

    prob = wl.random_problem(3, 2, 77, "magnus4_simpson", seed=14, g_norm=0.3)
    ctx = b.parament_create(0, None)
    try:
        H0 = np.ascontiguousarray(prob.H0)
        Hk = np.ascontiguousarray(prob.Hk)
        c = np.ascontiguousarray(prob.c)
        b.parament_set_hamiltonians(ctx, 3, 2, H0.ctypes.data, Hk.ctypes.data, b.PARAMENT_C128,
                                    b.PARAMENT_MAGNUS4_SIMPSON)
        b.parament_set_controls(ctx, c.ctypes.data, b.PARAMENT_F64, 77, prob.dt)
        U = np.zeros((3, 3), np.complex128)
        b.parament_propagate(ctx, U.ctypes.data, b.PARAMENT_PREC_FP64)
        assert np.max(np.abs(U - ref(prob))) <= TOL64
    finally:
        b.parament_destroy(ctx)


def test_state_machine_and_errors(prop, torch):
    from paper_2108_07126_gb300 import binding as b

    ctx = b.parament_create(0, None)
    try:
        U = torch.zeros(2, 2, dtype=torch.complex128, device="cuda")
        st = b.raw_call("parament_propagate", ctx, U.data_ptr(), 0)
        assert st == b.PARAMENT_ERR_STATE
        H = torch.tensor([[1.0, 2.0], [3.0, 1.0]], dtype=torch.complex128, device="cuda")  # not Hermitian
        st = b.raw_call("parament_set_hamiltonians", ctx, 2, 0, H.data_ptr(), None, 1, 0)
        assert st == b.PARAMENT_ERR_NOT_HERMITIAN
        Hn = torch.tensor([[float("nan"), 0.0], [0.0, 1.0]], dtype=torch.complex128, device="cuda")
        assert b.raw_call("parament_set_hamiltonians", ctx, 2, 0, Hn.data_ptr(), None, 1, 0) == b.PARAMENT_ERR_NONFINITE
        Hok = torch.eye(2, dtype=torch.complex128, device="cuda")
        assert b.raw_call("parament_set_hamiltonians", ctx, 0, 0, Hok.data_ptr(), None, 1, 0) == \
            b.PARAMENT_ERR_INVALID_VALUE
        assert b.raw_call("parament_set_hamiltonians", ctx, 257, 0, Hok.data_ptr(), None, 1, 0) == \
            b.PARAMENT_ERR_UNSUPPORTED
        assert b.raw_call("parament_set_controls", ctx, None, 1, 4, 0.1) == b.PARAMENT_ERR_STATE
        assert b.raw_call("parament_set_hamiltonians", ctx, 2, 0, Hok.data_ptr(), None, 1, 0) == b.PARAMENT_OK
        assert b.raw_call("parament_propagate", ctx, U.data_ptr(), 0) == b.PARAMENT_ERR_STATE
        assert b.raw_call("parament_set_controls", ctx, None, 1, -1, 0.1) == b.PARAMENT_ERR_INVALID_VALUE
        assert b.raw_call("parament_set_controls", ctx, None, 1, 4, 0.5) == b.PARAMENT_OK
        assert b.raw_call("parament_propagate", ctx, U.data_ptr(), 2) == b.PARAMENT_ERR_UNSUPPORTED
        assert b.raw_call("parament_propagate", ctx, U.data_ptr(), 0) == b.PARAMENT_OK
        torch.cuda.synchronize()
        ref_u = np.diag(np.exp(-1j * np.ones(2) * 2.0))
        assert np.max(np.abs(U.cpu().numpy() - ref_u)) <= TOL64
        assert b.raw_call("parament_set_option", ctx, 999, 0) == b.PARAMENT_ERR_INVALID_VALUE
        assert b.raw_call("parament_set_option", ctx, b.PARAMENT_OPT_TAYLOR_DEGREE, 5) == b.PARAMENT_ERR_INVALID_VALUE
    finally:
        b.parament_destroy(ctx)


def test_nonfinite_controls_flagged(prop):
    prob = wl.random_problem(4, 2, 40, "midpoint", seed=15)
    prob.c[1, 17] = np.nan
    run(prop, prob, "fp64")
    assert prop.stats()["device_status"] & 0x1


def test_mixed_control_dtypes(prop, torch):
    prob = wl.random_problem(4, 2, 200, "magnus4_gl2", seed=16, g_norm=0.3)
    U = run(prop, prob, "fp64", c_dtype=torch.float32)
    r = oracle.propagate(prob.H0, prob.Hk, prob.c.astype(np.float32).astype(np.float64), prob.dt, prob.integrator)
    assert np.max(np.abs(U - r)) <= TOL64
    U = run(prop, prob, "fp32", c_dtype=torch.float64, h_dtype=torch.complex128)
    check(np.max(np.abs(U - ref(prob))), tol32(4, 200))


# --- dimensions above 16: one thread block per leaf ------------------------------------------------


@pytest.mark.parametrize("integrator", INTEGRATORS)
@pytest.mark.parametrize("d", [17, 32, 40, 64, 100, 128, 192, 256])
def test_large_d_fp64_matches_oracle(prop, integrator, d):
    n = 37 if d <= 64 else (9 if d <= 128 else 5)
    prob = wl.random_problem(d, 2, n, integrator, seed=600 + d, g_norm=0.6)
    U = run(prop, prob, "fp64")
    assert np.max(np.abs(U - ref(prob))) <= TOL64


@pytest.mark.parametrize("d", [32, 64, 128, 192])
def test_large_d_fp32_matches_oracle(prop, d):
    n = 301 if d <= 64 else 41
    prob = wl.random_problem(d, 3, n, "magnus4_gl2", seed=700 + d, g_norm=0.5)
    U = run(prop, prob, "fp32")
    check(np.max(np.abs(U - ref32(prob))), tol32(d, n))


def run_stats(prop, prob, prec):
    import torch

    U = run(prop, prob, prec, c_dtype=torch.float32, h_dtype=torch.complex64)
    return U, prop.stats()


@pytest.mark.parametrize("d", [17, 32, 40, 64, 100, 128, 192, 256])
def test_tensor_core_tf32x3_matches_oracle(prop, d):
    """3xTF32 tensor-core products keep FP32 accuracy, on tcgen05 for every d > 16."""
    from paper_2108_07126_gb300 import binding as b

    n = 301 if d <= 64 else 41
    prob = wl.random_problem(d, 3, n, "magnus4_gl2", seed=900 + d, g_norm=0.5)
    U, st = run_stats(prop, prob, "fp32_tc_tf32x3")
    check(np.max(np.abs(U - ref32(prob))), tol_tc(d, n))
    assert st["product_backends"] == b.PARAMENT_BACKEND_TCGEN05
    assert st["device_status"] == 0


@pytest.mark.parametrize("d", [20, 32, 40, 64, 100, 128, 160, 256])
def test_tensor_core_bf16x3_matches_oracle(prop, d):
    """Split BF16x3 on tcgen05 (kind::f16, six products per real product) keeps FP32 accuracy."""
    from paper_2108_07126_gb300 import binding as b

    n = 301 if d <= 64 else 41
    prob = wl.random_problem(d, 3, n, "magnus4_gl2", seed=950 + d, g_norm=0.5)
    U, st = run_stats(prop, prob, "fp32_tc_bf16x3")
    check(np.max(np.abs(U - ref32(prob))), tol_tc(d, n))
    assert st["product_backends"] == b.PARAMENT_BACKEND_TCGEN05
    assert st["device_status"] == 0


@pytest.mark.parametrize("integrator", ["midpoint", "magnus4_simpson"])
@pytest.mark.parametrize("d,prec", [(32, "fp32_tc_tf32x3"), (64, "fp32_tc_bf16x3"), (64, "fp32_tc_tf32x3")])
def test_tensor_core_small_d_integrators(prop, integrator, d, prec):
    """The shared-memory tcgen05 body (d = 17..64) with the other two integrators and a norm range
    that needs squarings."""
    prob = wl.random_problem(d, 2, 257, integrator, seed=970 + d, g_norm=2.5)
    U, st = run_stats(prop, prob, prec)
    assert st["max_squarings"] >= 1
    check(np.max(np.abs(U - ref32(prob))), tol_tc(d, prob.n_steps))


@pytest.mark.parametrize("grid", [1, 3, 152, 304])
def test_tensor_core_small_d_tree_shapes(prop, grid):
    """Leaf lengths from 1 to the whole run: the same U(T) up to FP32 rounding."""
    from paper_2108_07126_gb300 import binding as b

    prob = wl.random_problem(48, 2, 400, "magnus4_gl2", seed=981, g_norm=0.5)
    prop.set_option(b.PARAMENT_OPT_GRID_BLOCKS, grid)
    U, st = run_stats(prop, prob, "fp32_tc_tf32x3")
    assert st["grid_blocks"] == min(grid, prob.n_steps)
    check(np.max(np.abs(U - ref32(prob))), tol_tc(48, prob.n_steps))


def test_product_backends_reported(prop):
    """parament_stats names the code that ran the products: CUDA cores for FP64, FP32 and d <= 16."""
    from paper_2108_07126_gb300 import binding as b

    for d, prec in ((8, "fp32"), (8, "fp64"), (64, "fp32"), (64, "fp64"), (128, "fp32")):
        prob = wl.random_problem(d, 2, 20, "midpoint", seed=990 + d, g_norm=0.3)
        run(prop, prob, prec)
        assert prop.stats()["product_backends"] == b.PARAMENT_BACKEND_CUDA_CORES, (d, prec)


def test_tensor_core_modes_rejected_where_not_built(prop, torch):
    from paper_2108_07126_gb300 import binding as b

    prob = wl.random_problem(16, 1, 10, "midpoint", seed=1)
    with pytest.raises(b.ParamentError) as e:
        run(prop, prob, "fp32_tc_tf32x3", c_dtype=torch.float32, h_dtype=torch.complex64)
    assert e.value.status == b.PARAMENT_ERR_UNSUPPORTED
    prob = wl.random_problem(300, 1, 4, "midpoint", seed=1)
    with pytest.raises(b.ParamentError) as e:
        run(prop, prob, "fp32_tc_bf16x3", c_dtype=torch.float32, h_dtype=torch.complex64)
    assert e.value.status == b.PARAMENT_ERR_UNSUPPORTED


@pytest.mark.parametrize("grid", [1, 2, 3, 7, 152])
def test_large_d_tree_shapes(prop, grid):
    from paper_2108_07126_gb300 import binding as b

    prob = wl.random_problem(48, 2, 200, "midpoint", seed=800, g_norm=0.3)
    prop.set_option(b.PARAMENT_OPT_GRID_BLOCKS, grid)
    U = run(prop, prob, "fp64")
    assert np.max(np.abs(U - ref(prob))) <= TOL64
    st = prop.stats()
    assert st["grid_blocks"] == min(grid, 200) and st["tree_products"] == 200


def test_large_d_big_norm_squarings(prop):
    prob = wl.random_problem(64, 1, 5, "midpoint", seed=801, g_norm=20.0)
    U = run(prop, prob, "fp64")
    assert np.max(np.abs(U - ref(prob))) <= 20 * TOL64
    assert prop.stats()["max_squarings"] >= 4


# --- the benchmark workloads -------------------------------------------------------------------


def test_rabi_qubit_full_size(prop):
    """Driven two-level system at N = 2^14: oracle parity, unitarity, RWA population."""
    prob = wl.rabi_qubit()
    U = run(prop, prob, "fp64")
    R = ref(prob)
    assert np.max(np.abs(U - R)) <= TOL64
    assert np.max(np.abs(U.conj().T @ U - np.eye(2))) <= 1e-12
    assert abs(U[1, 0]) ** 2 < 0.05
    U32 = run(prop, prob, "fp32")
    check(np.max(np.abs(U32 - R)), tol32(2, prob.n_steps))


def test_coupled_spins_slice_of_run(prop):
    """Four coupled spins, GL4, first 2^15 slices of the workload."""
    full = wl.coupled_spins(n_steps=1 << 15)
    U = run(prop, full, "fp64")
    R = ref(full)
    assert np.max(np.abs(U - R)) <= TOL64
    U32 = run(prop, full, "fp32", h_dtype=None)
    check(np.max(np.abs(U32 - ref32(full))), tol32(16, full.n_steps))


@pytest.mark.parametrize("d", [8, 40])
def test_host_controls_pinned_and_pageable(prop, torch, d):
    """Controls in page-locked host memory are read by the kernels in place, pageable host
    controls are copied first: both give bit-for-bit the U(T) of device-resident controls, and
    a host U_out receives it."""
    from paper_2108_07126_gb300 import binding as b

    prob = wl.random_problem(d, 3, 3000 if d <= 16 else 200, "magnus4_gl2", seed=4242 + d, g_norm=0.4)
    prop.set_hamiltonians(torch.as_tensor(prob.H0).to(torch.complex64), torch.as_tensor(prob.Hk).to(torch.complex64),
                          prob.integrator)
    c32 = torch.as_tensor(prob.c).to(torch.float32)
    prop.set_controls(c32.cuda(), prob.dt, prob.n_steps)
    U_dev = prop.propagate("fp32").cpu().numpy()
    pinned = c32.pin_memory()
    pageable = np.ascontiguousarray(c32.numpy())
    for ptr in (pinned.data_ptr(), pageable.ctypes.data):
        U_host = np.zeros((d, d), np.complex64)
        b.parament_set_controls(prop.ctx, ptr, b.PARAMENT_F32, prob.n_steps, prob.dt)
        b.parament_propagate(prop.ctx, U_host.ctypes.data, b.PARAMENT_PREC_FP32)
        assert np.array_equal(U_host, U_dev)


def test_dense_stress_full_size(prop, torch):
    """d = 128 dense stress at N = 2^16 in the benchmark's launch configuration: FP32, 3xTF32 and
    split BF16x3 stay unitary and agree with the FP64 path within the FP32 bound; the FP64 path
    is unitary; every precision matches the oracle on a 2^9-slice instance of the workload."""
    prob = wl.dense_stress()
    N, I = prob.n_steps, np.eye(128)
    U64 = run(prop, prob, "fp64")
    assert np.max(np.abs(U64.conj().T @ U64 - I)) <= 1e-10
    f32 = dict(c_dtype=torch.float32, h_dtype=torch.complex64)
    for prec in ("fp32", "fp32_tc_tf32x3", "fp32_tc_bf16x3"):
        U = run(prop, prob, prec, **f32)
        unit, err = np.max(np.abs(U.conj().T @ U - I)), np.max(np.abs(U - U64))
        check(unit, tol32(128, N) if prec == "fp32" else tol_tc(128, N), (prec, "unitarity"))
        check(err, FULL_SIZE["dense_stress"][prec], (prec, "vs FP64"))
    head = wl.dense_stress(n_steps=1 << 9)
    R = ref32(head)
    for prec in ("fp32", "fp32_tc_tf32x3", "fp32_tc_bf16x3"):
        check(np.max(np.abs(run(prop, head, prec, **f32) - R)), tol_tc(128, head.n_steps))


def test_fp32_unitary_step_removes_coherent_drift(prop):
    """Coupled spins, 2^18 slices: repeated FP32 rounding drifts U off the unitary group; one
    Newton-Schulz step per leaf product (the default) keeps it unitary and closer to the oracle."""
    from paper_2108_07126_gb300 import binding as b

    prob = wl.coupled_spins(n_steps=1 << 18)
    I = np.eye(16)
    out = {}
    for step in (0, 1):
        prop.set_option(b.PARAMENT_OPT_UNITARY_STEP, step)
        U = run(prop, prob, "fp32")
        out[step] = (np.max(np.abs(U.conj().T @ U - I)), U)
    U64 = run(prop, prob, "fp64")
    e0, e1 = (np.max(np.abs(out[s][1] - U64)) for s in (0, 1))
    assert out[1][0] < 1e-4 < out[0][0]
    assert e1 < e0
    check(e1, UNITARY_STEP_2_18, "with the step")


# --- the paper's Chebyshev exponential (Sec. 2.1, Algorithm 1) ------------------------------------


@pytest.mark.parametrize("integrator", INTEGRATORS)
@pytest.mark.parametrize("d", [2, 3, 8, 16])
def test_chebyshev_fp64_matches_oracle(prop, integrator, d):
    from paper_2108_07126_gb300 import binding as b

    prob = wl.random_problem(d, 2, 333, integrator, seed=1000 + d, g_norm=0.5)
    prop.set_option(b.PARAMENT_OPT_EXP_METHOD, 1)
    U = run(prop, prob, "fp64")
    assert np.max(np.abs(U - ref(prob))) <= TOL64
    st = prop.stats()
    # one product per degree and slice: exp_products = m N with m the global degree
    assert st["exp_products"] == st["max_degree"] * prob.n_steps and st["max_squarings"] == 0


@pytest.mark.parametrize("d", [4, 16])
def test_chebyshev_fp32_matches_oracle(prop, d):
    from paper_2108_07126_gb300 import binding as b

    prob = wl.random_problem(d, 3, 1000, "magnus4_gl2", seed=1100 + d, g_norm=0.4)
    prop.set_option(b.PARAMENT_OPT_EXP_METHOD, 1)
    U = run(prop, prob, "fp32")
    check(np.max(np.abs(U - ref32(prob))), tol32(d, prob.n_steps))


def test_chebyshev_degree_follows_the_bound(prop):
    """A larger spectral interval needs a higher Chebyshev degree (Table 1 grows with m)."""
    from paper_2108_07126_gb300 import binding as b

    degs = []
    for g in (0.05, 0.5, 3.0):
        prob = wl.random_problem(4, 1, 20, "midpoint", seed=1200, g_norm=g)
        prop.set_option(b.PARAMENT_OPT_EXP_METHOD, 1)
        U = run(prop, prob, "fp64")
        assert np.max(np.abs(U - ref(prob))) <= TOL64 * max(1.0, g)
        degs.append(prop.stats()["max_degree"])
    assert degs[0] < degs[1] < degs[2]


@pytest.mark.parametrize("integrator", INTEGRATORS)
@pytest.mark.parametrize("d", [20, 40, 100, 192])
def test_chebyshev_large_d_fp64_matches_oracle(prop, integrator, d):
    """The block-level kernel evaluates the Chebyshev series by Clenshaw with its own products."""
    from paper_2108_07126_gb300 import binding as b

    n = 23 if d <= 64 else 5
    prob = wl.random_problem(d, 2, n, integrator, seed=1300 + d, g_norm=0.6)
    prop.set_option(b.PARAMENT_OPT_EXP_METHOD, 1)
    U = run(prop, prob, "fp64")
    assert np.max(np.abs(U - ref(prob))) <= TOL64
    st = prop.stats()
    assert st["exp_products"] == st["max_degree"] * n and st["max_squarings"] == 0


@pytest.mark.parametrize("d,prec", [(32, "fp32"), (64, "fp32"), (128, "fp32"), (128, "fp32_tc_tf32x3"),
                                    (32, "fp32_tc_tf32x3"), (64, "fp32_tc_bf16x3")])
def test_chebyshev_large_d_fp32_matches_oracle(prop, d, prec):
    import torch

    from paper_2108_07126_gb300 import binding as b

    n = 101 if d <= 64 else 21
    prob = wl.random_problem(d, 3, n, "magnus4_gl2", seed=1400 + d, g_norm=0.5)
    prop.set_option(b.PARAMENT_OPT_EXP_METHOD, 1)
    U = run(prop, prob, prec, c_dtype=torch.float32, h_dtype=torch.complex64)
    check(np.max(np.abs(U - ref32(prob))), tol_tc(d, n))
