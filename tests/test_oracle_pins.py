"""Pins for the FP64 oracle: closed forms, convergence orders, brute force, invariants.

Each test checks the oracle against something other than itself -- a closed
form from the paper, a library routine that computes the same quantity by a
different method (scipy's Pade expm, an adaptive ODE solver), or finite
differences.  The planted-mistake tests show that a plausible slip in the
oracle (flipped commutator sign, reversed product order, dropped Omega_2,
dropped conj) makes one of the pins fail.
"""

import json
import math
import os

import numpy as np
import pytest
import scipy.integrate
import scipy.linalg

import oracle
import oracle.parament_oracle as orc
from paper_2108_07126_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
INTEGRATORS = ("midpoint", "magnus4_gl2", "magnus4_simpson")


def _circular_params():
    with open(os.path.join(GOLDEN, "circular_drive.json")) as f:
        return json.load(f)


def circular_exact(w0, w1, wrf, t):
    """Closed-form propagator of the circular drive (rotating frame, Sec. 5).

    H(t) = R(t) H_r R(t)^dagger with R(t) = exp(-i wrf t sz/2) and
    H_r = (w0/2) sz + (w1/2) sx, so U(t) = R(t) exp(-i t [(w0 - wrf)/2 sz + w1/2 sx]).
    """
    R = scipy.linalg.expm(-0.5j * wrf * t * wl.SZ)
    return R @ scipy.linalg.expm(-1j * t * (0.5 * (w0 - wrf) * wl.SZ + 0.5 * w1 * wl.SX))


def circular_error(integrator, n_steps, p=None):
    p = p or _circular_params()
    prob = wl.circular_drive(n_steps, integrator, p["w0"], p["w1"], p["w_rf"], p["t_final"])
    U = oracle.propagate(prob.H0, prob.Hk, prob.c, prob.dt, integrator)
    return np.max(np.abs(U - circular_exact(p["w0"], p["w1"], p["w_rf"], p["t_final"])))


def observed_order(integrator, n_list=(24, 48, 96)):
    errs = [circular_error(integrator, n) for n in n_list]
    return [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)], errs


# --- static Hamiltonian: exact exp(-i H T) -------------------------------------------------


@pytest.mark.parametrize("integrator", INTEGRATORS)
def test_static_hamiltonian_is_exact(integrator):
    rng = np.random.default_rng(1)
    d, K, N, dt = 5, 2, 7, 0.37
    H0 = wl.random_hermitian(rng, d)
    Hk = np.stack([wl.random_hermitian(rng, d) for _ in range(K)])
    amp = rng.standard_normal(K)
    c = np.repeat(amp[:, None], wl.n_samples(N, integrator), axis=1)
    U = oracle.propagate(H0, Hk, c, dt, integrator)
    H = H0 + np.einsum("k,kab->ab", amp, Hk)
    ref = scipy.linalg.expm(-1j * H * (N * dt))
    assert np.max(np.abs(U - ref)) < 1e-12


@pytest.mark.parametrize("norm", [1e-3, 0.2, 1.0, 8.0, 40.0])
def test_slice_exponential_matches_pade(norm):
    rng = np.random.default_rng(2)
    G = np.stack([wl.gue(rng, 7, norm) for _ in range(4)])
    U = oracle.exact_slice_propagators(G)
    ref = np.stack([scipy.linalg.expm(-1j * g) for g in G])
    assert np.max(np.abs(U - ref)) < 2e-13 * max(1.0, norm)


# --- ordering -----------------------------------------------------------------------------


@pytest.mark.parametrize("n", [0, 1, 2, 3, 5, 6, 67, 128, 129])
def test_tree_equals_time_ordered_product(n):
    rng = np.random.default_rng(3)
    d = 3
    U = np.stack([wl.haar_unitary(rng, d) for _ in range(n)]) if n else np.zeros((0, d, d), np.complex128)
    ref = np.eye(d, dtype=np.complex128)
    for j in range(n):
        ref = U[j] @ ref  # later slices multiply from the left (Eq. slices)
    assert np.max(np.abs(oracle.ordered_product(U) - ref)) < 1e-13


# --- the paper's convergence example (Sec. 5, Fig. 4) -------------------------------------


@pytest.mark.parametrize("integrator", INTEGRATORS)
def test_circular_drive_convergence_order(integrator):
    p = _circular_params()
    slopes, errs = observed_order(integrator)
    want = p["order"][integrator]
    for s in slopes:
        assert abs(s - want) < 0.1, (slopes, errs)


def test_circular_drive_converges_to_closed_form():
    # fourth-order methods reach ~1e-12 with a few thousand steps per the FP64 regime of Fig. 4
    assert circular_error("magnus4_gl2", 4096) < 1e-11
    assert circular_error("magnus4_simpson", 4096) < 1e-11
    assert circular_error("midpoint", 4096) < 5e-7


def test_resonant_rabi_population():
    # w0 = w_rf: the rotating-frame Hamiltonian is (w1/2) sx, so P_1(t) = sin^2(w1 t / 2) exactly
    w1, t = 0.1, 6.0
    prob = wl.circular_drive(2048, "magnus4_gl2", 1.0, w1, 1.0, t)
    U = oracle.propagate(prob.H0, prob.Hk, prob.c, prob.dt, prob.integrator)
    P1 = abs(U[1, 0]) ** 2
    assert abs(P1 - math.sin(0.5 * w1 * t) ** 2) < 1e-12


def test_rabi_workload_rwa_population():
    # linear drive at resonance, T = 1 us: RWA predicts P_1 = sin^2(Omega T / 2) = 0 (10 Rabi cycles);
    # the counter-rotating term and the 61 ps step leave a small deviation (a loose sanity bound)
    prob = wl.rabi_qubit()
    U = oracle.propagate(prob.H0, prob.Hk, prob.c, prob.dt, prob.integrator)
    assert abs(U[1, 0]) ** 2 < 0.05
    # pi pulse: in the rotating-wave limit H_eff = (Omega/2) sx, so P_1 = sin^2(Omega t / 2) and T_pi = pi / Omega
    T_pi = math.pi / prob.meta["Omega"]
    n_pi = 4096
    prob_pi = wl.rabi_qubit(n_pi, T_pi)
    U = oracle.propagate(prob_pi.H0, prob_pi.Hk, prob_pi.c, prob_pi.dt, prob_pi.integrator)
    assert abs(U[1, 0]) ** 2 > 0.99


# --- trajectories: the propagator at every intermediate time -------------------------------


@pytest.mark.parametrize("integrator", INTEGRATORS)
def test_trajectory_static_hamiltonian_is_exact_at_every_time(integrator):
    # all c constant: U(t_n) = exp(-i H n dt) at every output time, for any stride
    rng = np.random.default_rng(11)
    d, K, N, dt = 4, 2, 13, 0.21
    H0 = wl.random_hermitian(rng, d)
    Hk = np.stack([wl.random_hermitian(rng, d) for _ in range(K)])
    amp = rng.standard_normal(K)
    c = np.repeat(amp[:, None], wl.n_samples(N, integrator), axis=1)
    H = H0 + np.einsum("k,kab->ab", amp, Hk)
    for every in (1, 4, 13, 20):
        times = oracle.trajectory_times(N, every)
        traj = oracle.trajectory(H0, Hk, c, dt, integrator, every)
        assert traj.shape == (len(times), d, d)
        for n, U in zip(times, traj):
            assert np.max(np.abs(U - scipy.linalg.expm(-1j * H * (n * dt)))) < 1e-12


def test_trajectory_times_cover_the_last_slice():
    assert list(oracle.trajectory_times(10, 3)) == [3, 6, 9, 10]
    assert list(oracle.trajectory_times(9, 3)) == [3, 6, 9]
    assert list(oracle.trajectory_times(5, 1)) == [1, 2, 3, 4, 5]
    assert list(oracle.trajectory_times(4, 7)) == [4]
    assert len(oracle.trajectory_times(0, 2)) == 0


@pytest.mark.parametrize("integrator", ["magnus4_gl2", "magnus4_simpson"])
def test_trajectory_follows_circular_drive_closed_form(integrator):
    # every intermediate U(t_n) against the closed form of the circular drive (Sec. 5)
    p = _circular_params()
    N, every = 2048, 64
    prob = wl.circular_drive(N, integrator, p["w0"], p["w1"], p["w_rf"], p["t_final"])
    traj = oracle.trajectory(prob.H0, prob.Hk, prob.c, prob.dt, integrator, every)
    for n, U in zip(oracle.trajectory_times(N, every), traj):
        ref = circular_exact(p["w0"], p["w1"], p["w_rf"], n * prob.dt)
        assert np.max(np.abs(U - ref)) < 1e-10


def test_trajectory_resonant_rabi_population_over_time():
    # w0 = w_rf: P_1(t) = sin^2(w1 t / 2) at every output time; states from psi0 = |0>
    w1, t = 0.1, 40.0
    N, every = 4000, 100
    prob = wl.circular_drive(N, "magnus4_gl2", 1.0, w1, 1.0, t)
    psi = oracle.trajectory(prob.H0, prob.Hk, prob.c, prob.dt, prob.integrator, every, psi0=np.array([1.0, 0.0]))
    times = oracle.trajectory_times(N, every) * prob.dt
    P1 = np.abs(psi[:, 1]) ** 2
    assert np.max(np.abs(P1 - np.sin(0.5 * w1 * times) ** 2)) < 1e-10
    assert P1.max() > 0.99  # a full Rabi flop happens inside the window


def test_trajectory_last_entry_is_the_tree_product():
    # sequential prefix products end at the pairwise-tree U(T) (two orders of evaluation)
    prob = wl.random_problem(5, 3, 37, "magnus4_gl2", seed=12, g_norm=0.8)
    traj = oracle.trajectory(prob.H0, prob.Hk, prob.c, prob.dt, prob.integrator, 5)
    U = oracle.propagate(prob.H0, prob.Hk, prob.c, prob.dt, prob.integrator)
    assert np.max(np.abs(traj[-1] - U)) < 1e-13
    psi0 = wl.haar_unitary(np.random.default_rng(13), 5)[:, 0]
    psi = oracle.trajectory(prob.H0, prob.Hk, prob.c, prob.dt, prob.integrator, 5, psi0=psi0)
    assert np.max(np.abs(psi - traj @ psi0)) < 1e-14


def _circular_trajectory_error(fn_traj, every=256, N=1024):
    p = _circular_params()
    prob = wl.circular_drive(N, "magnus4_gl2", p["w0"], p["w1"], p["w_rf"], p["t_final"])
    traj = fn_traj(prob.H0, prob.Hk, prob.c, prob.dt, prob.integrator, every)
    return max(np.max(np.abs(U - circular_exact(p["w0"], p["w1"], p["w_rf"], n * prob.dt)))
               for n, U in zip(oracle.trajectory_times(N, every), traj))


def test_planted_transposed_slices_fail_trajectory_closed_form(monkeypatch):
    # a row/column-major mix-up of the slice propagators (U_j^T) breaks the intermediate closed forms
    assert _circular_trajectory_error(orc.trajectory) < 1e-8
    real = orc.exact_slice_propagators
    monkeypatch.setattr(orc, "exact_slice_propagators", lambda G: np.swapaxes(real(G), -1, -2))
    assert _circular_trajectory_error(orc.trajectory) > 1e-3


def test_planted_off_by_one_output_time_fails_closed_form(monkeypatch):
    # keeping R one slice early (after slice n - 1 instead of n) is caught at the step size
    real = orc.trajectory_times
    monkeypatch.setattr(orc, "trajectory_times", lambda n, every: real(n, every) - 1)
    assert _circular_trajectory_error(orc.trajectory) > 1e-4


# --- brute-force ODE integration ---------------------------------------------------------


def _ode_propagator(Hfun, t0, t1, d, U0):
    def rhs(t, y):
        U = y.reshape(d, d)
        return (-1j * Hfun(t) @ U).ravel()

    sol = scipy.integrate.solve_ivp(rhs, (t0, t1), U0.ravel(), method="DOP853", rtol=1e-13, atol=1e-13)
    return sol.y[:, -1].reshape(d, d)


def test_piecewise_constant_controls_match_ode():
    # for controls constant on each slice the midpoint propagator is the exact solution
    rng = np.random.default_rng(4)
    d, K, N, dt = 3, 2, 5, 0.4
    H0 = wl.random_hermitian(rng, d)
    Hk = np.stack([wl.random_hermitian(rng, d) for _ in range(K)])
    c = rng.standard_normal((K, N))
    U = np.eye(d, dtype=np.complex128)
    for j in range(N):
        Hj = H0 + np.einsum("k,kab->ab", c[:, j], Hk)
        U = _ode_propagator(lambda t, Hj=Hj: Hj, j * dt, (j + 1) * dt, d, U)
    assert np.max(np.abs(oracle.propagate(H0, Hk, c, dt, "midpoint") - U)) < 1e-11
    # Gauss-Legendre with equal node samples reduces to the midpoint exponent
    c2 = np.repeat(c, 2, axis=1)
    assert np.max(np.abs(oracle.propagate(H0, Hk, c2, dt, "magnus4_gl2") - U)) < 1e-11


@pytest.mark.parametrize("integrator,order", [("midpoint", 2), ("magnus4_gl2", 4), ("magnus4_simpson", 4)])
def test_smooth_controls_converge_to_ode(integrator, order):
    rng = np.random.default_rng(5)
    d, K, T = 4, 2, 3.0
    H0 = wl.random_hermitian(rng, d, 0.7)
    Hk = np.stack([wl.random_hermitian(rng, d, 0.7) for _ in range(K)])
    freq = rng.uniform(0.5, 2.0, K)
    phase = rng.uniform(0, 2 * math.pi, K)

    def ctrl(t):
        return np.cos(freq[:, None] * np.atleast_1d(t)[None, :] + phase[:, None])

    ref = _ode_propagator(lambda t: H0 + np.einsum("k,kab->ab", ctrl(t)[:, 0], Hk), 0.0, T, d,
                          np.eye(d, dtype=np.complex128))
    errs = []
    for N in (16, 32, 64):
        dt = T / N
        c = ctrl(wl.sample_times(N, dt, integrator))
        errs.append(np.max(np.abs(oracle.propagate(H0, Hk, c, dt, integrator) - ref)))
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(s - order) < 0.3 for s in slopes), (slopes, errs)


# --- invariants ---------------------------------------------------------------------------


@pytest.mark.parametrize("integrator", INTEGRATORS)
def test_unitarity_and_determinant(integrator):
    prob = wl.random_problem(6, 3, 101, integrator, seed=6, g_norm=0.5)
    U = oracle.propagate(prob.H0, prob.Hk, prob.c, prob.dt, integrator)
    assert np.max(np.abs(U.conj().T @ U - np.eye(6))) < 1e-13
    G = oracle.slice_exponents(prob.H0, prob.Hk, prob.c, prob.dt, integrator)
    # det U = prod_j det exp(-i G_j) = exp(-i sum_j Tr G_j)
    assert abs(np.linalg.det(U) - np.exp(-1j * np.trace(G, axis1=1, axis2=2).sum())) < 1e-12
    assert np.allclose(G, np.conj(np.swapaxes(G, 1, 2)), atol=1e-15)


def test_effective_control_count():
    # Sec. 4: N controls map to 3/2 N + N^2/2 effective controls
    for K in range(0, 10):
        assert oracle.effective_control_count(K) == (3 * K + K * K) // 2
    assert oracle.effective_control_count(8) == 44
    assert oracle.effective_control_count(4) == 14


# --- gradient -----------------------------------------------------------------------------


def _fd_gradient(prob, V, h, entries, integrator="midpoint"):
    out = []
    for (k, j) in entries:
        cp = prob.c.copy()
        cm = prob.c.copy()
        cp[k, j] += h
        cm[k, j] -= h
        Lp = oracle.gate_loss(oracle.propagate(prob.H0, prob.Hk, cp, prob.dt, integrator), V)
        Lm = oracle.gate_loss(oracle.propagate(prob.H0, prob.Hk, cm, prob.dt, integrator), V)
        out.append((Lp - Lm) / (2 * h))
    return np.array(out)


def test_frechet_matches_block_exponential():
    # Van Loan: exp([[X, E], [0, X]]) has L_X(E) in its upper-right block
    rng = np.random.default_rng(7)
    d = 5
    G = wl.random_hermitian(rng, d, 0.8)
    E = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    X = -1j * G
    blk = np.zeros((2 * d, 2 * d), np.complex128)
    blk[:d, :d] = X
    blk[d:, d:] = X
    blk[:d, d:] = E
    ref = scipy.linalg.expm(blk)[:d, d:]
    assert np.max(np.abs(oracle.frechet_exp(G, E) - ref)) < 1e-13
    # degenerate spectrum: the divided difference reduces to the derivative
    Gd = np.diag([0.3, 0.3, -0.2, 0.3, 1.1]).astype(np.complex128)
    blk[:d, :d] = -1j * Gd
    blk[d:, d:] = -1j * Gd
    ref = scipy.linalg.expm(blk)[:d, d:]
    assert np.max(np.abs(oracle.frechet_exp(Gd, E) - ref)) < 1e-13


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(8)
    prob = wl.random_problem(4, 3, 12, "midpoint", seed=8, g_norm=0.4)
    V = wl.haar_unitary(rng, 4)
    loss, grad, U = oracle.loss_and_gradient(prob.H0, prob.Hk, prob.c, prob.dt, V)
    assert abs(loss - oracle.gate_loss(U, V)) < 1e-15
    entries = [(k, j) for k in range(3) for j in range(12)]
    fd = _fd_gradient(prob, V, 1e-6, entries)
    g = np.array([grad[k, j] for (k, j) in entries])
    assert np.max(np.abs(g - fd)) <= 1e-6 * np.max(np.abs(fd))


def test_gradient_workload_subset_matches_fd():
    prob = wl.gradient_qubits(n_steps=256)
    loss, grad, U = oracle.loss_and_gradient(prob.H0, prob.Hk, prob.c, prob.dt, prob.V)
    rng = np.random.default_rng(9)
    entries = [(int(rng.integers(0, 6)), int(rng.integers(0, 256))) for _ in range(16)]
    fd = _fd_gradient(prob, prob.V, 1e-6, entries)
    g = np.array([grad[k, j] for (k, j) in entries])
    assert np.max(np.abs(g - fd)) <= 1e-6 * np.max(np.abs(fd))


@pytest.mark.parametrize("integrator", ["magnus4_gl2", "magnus4_simpson"])
def test_magnus_gradient_matches_finite_differences(integrator):
    # every sample of a short run, including the Simpson end points shared by two slices
    rng = np.random.default_rng(21)
    prob = wl.random_problem(3, 2, 7, integrator, seed=21, g_norm=0.5)
    V = wl.haar_unitary(rng, 3)
    loss, grad, U = oracle.loss_and_gradient(prob.H0, prob.Hk, prob.c, prob.dt, V, integrator)
    assert grad.shape == prob.c.shape
    assert abs(loss - oracle.gate_loss(oracle.propagate(prob.H0, prob.Hk, prob.c, prob.dt, integrator), V)) < 1e-14
    entries = [(k, s) for k in range(2) for s in range(prob.c.shape[1])]
    fd = _fd_gradient(prob, V, 1e-6, entries, integrator)
    g = np.array([grad[k, s] for (k, s) in entries])
    assert np.max(np.abs(g - fd)) <= 1e-6 * np.max(np.abs(fd))


def test_magnus_gradient_reduces_to_midpoint_for_equal_nodes():
    # GL4 with c1 = c2 per slice: the commutator term and its derivative vanish, G = dt H, and
    # dL/dc1 + dL/dc2 equals the midpoint gradient of the same piecewise-constant controls
    rng = np.random.default_rng(22)
    mid = wl.random_problem(4, 2, 9, "midpoint", seed=22, g_norm=0.4)
    c2 = np.repeat(mid.c, 2, axis=1)
    V = wl.haar_unitary(rng, 4)
    _, g_mid, U_mid = oracle.loss_and_gradient(mid.H0, mid.Hk, mid.c, mid.dt, V, "midpoint")
    _, g_gl, U_gl = oracle.loss_and_gradient(mid.H0, mid.Hk, c2, mid.dt, V, "magnus4_gl2")
    assert np.max(np.abs(U_mid - U_gl)) < 1e-13
    assert np.max(np.abs(g_gl[:, 0::2] + g_gl[:, 1::2] - g_mid)) < 1e-13


def test_planted_commutator_derivative_sign_fails_fd(monkeypatch):
    # a sign slip in the derivative of the Omega_2 term (i w [H_k, H2] -> -i w [H_k, H2])
    real = orc.exponent_derivatives

    def planted(H0, Hk, c, dt, integrator):
        out = real(H0, Hk, c, dt, integrator)
        Hk_ = np.asarray(Hk, dtype=np.complex128)
        return [(off, 2 * (0.5 * dt) * Hk_[None] - D) if off == 0 else (off, D) for off, D in out]

    monkeypatch.setattr(orc, "exponent_derivatives", planted)
    rng = np.random.default_rng(23)
    prob = wl.random_problem(3, 2, 5, "magnus4_gl2", seed=23, g_norm=0.8)
    V = wl.haar_unitary(rng, 3)
    _, grad, _ = orc.loss_and_gradient(prob.H0, prob.Hk, prob.c, prob.dt, V, "magnus4_gl2")
    monkeypatch.undo()
    entries = [(k, s) for k in range(2) for s in range(0, 10, 2)]
    fd = _fd_gradient(prob, V, 1e-6, entries, "magnus4_gl2")
    g = np.array([grad[k, s] for (k, s) in entries])
    assert np.max(np.abs(g - fd)) > 1e-4 * np.max(np.abs(fd))


def test_gradient_invariants():
    rng = np.random.default_rng(10)
    d = 4
    prob = wl.random_problem(d, 2, 9, "midpoint", seed=10, g_norm=0.4)
    Hk = np.concatenate([prob.Hk, np.eye(d, dtype=np.complex128)[None]])
    c = np.concatenate([prob.c, rng.standard_normal((1, 9))])
    V = wl.haar_unitary(rng, d)
    loss, grad, U = oracle.loss_and_gradient(prob.H0, Hk, c, prob.dt, V)
    # a control along the identity only changes the global phase, which L ignores
    assert np.max(np.abs(grad[-1])) < 1e-14
    assert 0.0 <= loss <= 1.0
    loss_u, grad_u, _ = oracle.loss_and_gradient(prob.H0, Hk, c, prob.dt, U)
    assert abs(loss_u) < 1e-14
    assert np.max(np.abs(grad_u)) < 1e-12  # V = U is a minimum


# --- planted mistakes: each must break a pin ------------------------------------------------


def test_planted_commutator_sign_breaks_fourth_order(monkeypatch):
    # the sign printed with the Simpson exponent: Omega_2 enters with the opposite sign
    monkeypatch.setattr(orc, "commutator", lambda A, B: B @ A - A @ B)
    for integrator in ("magnus4_gl2", "magnus4_simpson"):
        slopes, _ = observed_order(integrator)
        assert all(abs(s - 2.0) < 0.2 for s in slopes)


def test_planted_missing_omega2_stays_second_order(monkeypatch):
    # Sec. 5: higher quadrature order for Omega_1 alone does not improve convergence
    monkeypatch.setattr(orc, "commutator", lambda A, B: np.zeros_like(A))
    slopes, _ = observed_order("magnus4_simpson")
    assert all(abs(s - 2.0) < 0.2 for s in slopes)


def test_planted_reversed_product_order_fails_closed_form(monkeypatch):
    real = orc.ordered_product
    monkeypatch.setattr(orc, "ordered_product", lambda U: real(U[::-1]))
    assert circular_error("magnus4_gl2", 4096) > 1e-3


def test_planted_gradient_without_conj_fails_fd(monkeypatch):
    real_conj = np.conj
    rng = np.random.default_rng(8)
    prob = wl.random_problem(4, 3, 12, "midpoint", seed=8, g_norm=0.4)
    V = wl.haar_unitary(rng, 4)
    _, grad_ok, _ = oracle.loss_and_gradient(prob.H0, prob.Hk, prob.c, prob.dt, V)
    # plant: the gradient formula without conj(z) (np.conj on a scalar returns it unchanged)
    monkeypatch.setattr(orc.np, "conj", lambda x: x if np.ndim(x) == 0 else real_conj(x))
    _, grad_bad, _ = orc.loss_and_gradient(prob.H0, prob.Hk, prob.c, prob.dt, V)
    monkeypatch.undo()
    entries = [(k, j) for k in range(3) for j in range(12)]
    fd = _fd_gradient(prob, V, 1e-6, entries)
    g_bad = np.array([grad_bad[k, j] for (k, j) in entries])
    g_ok = np.array([grad_ok[k, j] for (k, j) in entries])
    assert np.max(np.abs(g_ok - fd)) <= 1e-6 * np.max(np.abs(fd))
    assert np.max(np.abs(g_bad - fd)) > 1e-3 * np.max(np.abs(fd))


@pytest.mark.parametrize("integrator", ["midpoint", "magnus4_gl2", "magnus4_simpson"])
def test_parallel_oracle_equals_single_process(integrator):
    """The multi-process oracle (contiguous slice ranges, partial products in time order) gives the
    single-process oracle's U(T) up to FP64 rounding, for every integrator's sample layout."""
    from oracle.parallel import propagate_parallel

    prob = wl.random_problem(5, 2, 301, integrator, seed=1234, g_norm=0.4)
    U1 = oracle.propagate(prob.H0, prob.Hk, prob.c, prob.dt, prob.integrator)
    U4 = propagate_parallel(prob.H0, prob.Hk, prob.c, prob.dt, prob.integrator, workers=4)
    assert np.max(np.abs(U1 - U4)) <= 1e-13
