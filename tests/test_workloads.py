"""The seeded synthetic inputs match the recipe each benchmark workload states (CPU only).

Each workload is checked against its own description: shapes and sample counts per integrator,
Hermitian operators with the stated spectra or spectral norms, control amplitudes in the
stated ranges, and the same arrays for the same seed.  Nothing here runs the method.
"""

import math

import numpy as np
import pytest

from paper_2108_07126_gb300 import workloads as wl

TWO_PI = 2.0 * math.pi


def hermitian(A, tol=1e-12):
    return np.max(np.abs(A - A.conj().T)) <= tol * max(1.0, np.max(np.abs(A)))


@pytest.mark.parametrize("integrator,extra", [("midpoint", 0), ("magnus4_gl2", 0), ("magnus4_simpson", 1)])
def test_sample_counts_per_integrator(integrator, extra):
    n = 37
    per = 1 if integrator == "midpoint" else 2
    assert wl.n_samples(n, integrator) == per * n + extra
    t = wl.sample_times(n, 0.5, integrator)
    assert t.shape == (per * n + extra,) and np.all(np.diff(t) > 0)
    assert 0.0 <= t[0] and t[-1] <= n * 0.5 + 1e-12


def test_gue_and_haar():
    rng = np.random.default_rng(3)
    for d in (2, 7, 64):
        H = wl.gue(rng, d, 2.5)
        assert hermitian(H) and abs(np.max(np.abs(np.linalg.eigvalsh(H))) - 2.5) < 1e-12
        V = wl.haar_unitary(rng, d)
        assert np.max(np.abs(V.conj().T @ V - np.eye(d))) < 1e-12


def test_rabi_qubit_recipe():
    p = wl.rabi_qubit()
    assert p.dim == 2 and p.n_steps == 1 << 14 and p.integrator == "midpoint"
    assert abs(p.dt * p.n_steps - 1000.0) < 1e-9  # T = 1 us in ns
    assert np.allclose(np.linalg.eigvalsh(p.H0), [-TWO_PI / 2, TWO_PI / 2])  # w0 = 2 pi * 1 GHz
    assert p.c.shape == (1, 1 << 14) and abs(np.max(np.abs(p.c)) - TWO_PI * 0.01) < 1e-4


def test_coupled_spins_recipe():
    p = wl.coupled_spins(n_steps=4096)
    assert p.dim == 16 and p.Hk.shape == (8, 16, 16) and p.integrator == "magnus4_gl2"
    assert p.c.shape == (8, 2 * 4096) and p.dt == 0.01
    assert hermitian(p.H0) and all(hermitian(h) for h in p.Hk)
    assert np.max(np.abs(p.H0 - np.diag(np.diag(p.H0)))) == 0.0  # Zeeman + ZZ: diagonal
    w = np.array(p.meta["w"])
    assert np.all((w >= TWO_PI * 0.5) & (w <= TWO_PI * 1.5))
    assert np.all((np.array(p.meta["J"]) >= 1e-3) & (np.array(p.meta["J"]) <= 10e-3))
    assert np.max(np.abs(p.c)) <= 3 * TWO_PI * 0.01  # three sinusoids of amplitude <= 2 pi 10 MHz
    # Pauli controls: sx_i, sy_i have eigenvalues +-1
    assert all(np.allclose(np.abs(np.linalg.eigvalsh(h)), 1.0) for h in p.Hk)


def test_gradient_qubits_recipe():
    p = wl.gradient_qubits(n_steps=2048)
    assert p.dim == 8 and p.Hk.shape == (6, 8, 8) and p.c.shape == (6, 2048) and p.dt == 1.0
    assert np.max(np.abs(p.V.conj().T @ p.V - np.eye(8))) < 1e-12
    assert abs(np.std(p.c) / (TWO_PI * 0.02) - 1.0) < 0.05  # N(0, (2 pi 20 MHz)^2)
    assert np.max(np.abs(np.diag(p.H0))) <= 0.5 * 3 * TWO_PI * 5e-3 + 2 * TWO_PI * 10e-3 / 4


def test_batched_instances_recipe():
    probs = wl.batched_instances()
    assert len(probs) == 256
    assert {p.dim for p in probs} == {2, 4, 8, 16, 32, 64}
    Ns = np.array([p.n_steps for p in probs])
    assert Ns.min() >= 1000 and Ns.max() <= 100000
    assert 2 <= min(p.Hk.shape[0] for p in probs) and max(p.Hk.shape[0] for p in probs) <= 6
    for p in probs[:12]:
        assert abs(np.max(np.abs(np.linalg.eigvalsh(p.H0))) - TWO_PI) < 1e-9
        assert all(abs(np.max(np.abs(np.linalg.eigvalsh(h))) - 1.0) < 1e-12 for h in p.Hk)
        assert p.c.shape == (p.Hk.shape[0], p.n_steps) and p.integrator == "midpoint"
    # log-uniform N: about half of the instances below sqrt(1e3 * 1e5) = 1e4
    assert 0.35 < np.mean(Ns < 1e4) < 0.65


def test_dense_stress_recipe():
    p = wl.dense_stress(n_steps=512)
    assert p.dim == 128 and p.Hk.shape == (4, 128, 128) and p.c.shape == (4, 1024)
    assert abs(np.max(np.abs(np.linalg.eigvalsh(p.H0))) - TWO_PI * 0.1) < 1e-12
    assert abs(p.dt - 0.2 / (TWO_PI * 0.1)) < 1e-15


def test_seeded_inputs_repeat():
    a, b = wl.dense_stress(n_steps=64), wl.dense_stress(n_steps=64)
    assert np.array_equal(a.H0, b.H0) and np.array_equal(a.c, b.c)
    a, b = wl.random_problem(5, 2, 10, seed=9), wl.random_problem(5, 2, 10, seed=9)
    assert np.array_equal(a.Hk, b.Hk) and np.array_equal(a.c, b.c)
