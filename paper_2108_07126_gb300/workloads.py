"""Seeded synthetic inputs for the propagator (numpy only).

This module only builds input arrays -- Hamiltonians, control samples,
target gates -- and holds none of the propagation arithmetic.  Both the CUDA
library's tests and the FP64 oracle consume the arrays it returns.

Units: time in ns, angular frequency in rad/ns (so 2*pi*1 GHz = 2*pi rad/ns).
The exponent G = H * dt is unit-free and identical to the SI form.

Sample positions follow the interface convention of the library (the same
one the oracle takes): midpoint -- one sample per slice at t_j + dt/2;
Gauss-Legendre -- two per slice at t_j + dt (1/2 -+ sqrt(3)/6); Simpson --
2N + 1 samples at multiples of dt/2.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

TWO_PI = 2.0 * math.pi
SEED_BASE = 20210816

SX = np.array([[0, 1], [1, 0]], dtype=np.complex128)
SY = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
SZ = np.array([[1, 0], [0, -1]], dtype=np.complex128)
I2 = np.eye(2, dtype=np.complex128)

INTEGRATOR_NAMES = ("midpoint", "magnus4_gl2", "magnus4_simpson")


@dataclasses.dataclass
class Problem:
    """One propagation problem: H0 (d,d), Hk (K,d,d), c (K,S), dt, integrator."""

    name: str
    H0: np.ndarray
    Hk: np.ndarray
    c: np.ndarray
    dt: float
    integrator: str
    n_steps: int
    V: np.ndarray | None = None
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def dim(self) -> int:
        return self.H0.shape[0]

    @property
    def n_ctrl(self) -> int:
        return self.Hk.shape[0]


def n_samples(n_steps: int, integrator: str) -> int:
    return {"midpoint": n_steps, "magnus4_gl2": 2 * n_steps,
            "magnus4_simpson": 2 * n_steps + 1}[integrator]


def sample_times(n_steps: int, dt: float, integrator: str) -> np.ndarray:
    """Times at which control samples are expected (interface convention)."""
    j = np.arange(n_steps, dtype=np.float64)
    if integrator == "midpoint":
        return (j + 0.5) * dt
    if integrator == "magnus4_gl2":
        off = math.sqrt(3.0) / 6.0
        t = np.empty(2 * n_steps)
        t[0::2] = (j + 0.5 - off) * dt
        t[1::2] = (j + 0.5 + off) * dt
        return t
    if integrator == "magnus4_simpson":
        return np.arange(2 * n_steps + 1, dtype=np.float64) * (0.5 * dt)
    raise ValueError(integrator)


def embed(op: np.ndarray, site: int, n_sites: int) -> np.ndarray:
    """op acting on ``site`` of ``n_sites`` qubits; qubit 0 is the most significant."""
    out = np.ones((1, 1), dtype=np.complex128)
    for s in range(n_sites):
        out = np.kron(out, op if s == site else I2)
    return out


def gue(rng: np.random.Generator, d: int, spectral_norm: float) -> np.ndarray:
    """Random Hermitian matrix (A + A^dagger)/2, A complex Gaussian, rescaled to a spectral norm."""
    A = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    H = 0.5 * (A + A.conj().T)
    return H * (spectral_norm / np.max(np.abs(np.linalg.eigvalsh(H))))


def haar_unitary(rng: np.random.Generator, d: int) -> np.ndarray:
    """Haar-random unitary: QR of a complex Ginibre matrix, phases of diag(R) divided out (Mezzadri 2007)."""
    Z = (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) / math.sqrt(2.0)
    Q, R = np.linalg.qr(Z)
    ph = np.diag(R) / np.abs(np.diag(R))
    return Q * ph[None, :]


def random_hermitian(rng: np.random.Generator, d: int, scale: float = 1.0) -> np.ndarray:
    A = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    return scale * 0.5 * (A + A.conj().T)


def random_problem(d: int, K: int, n_steps: int, integrator: str = "midpoint", seed: int = 0,
                   g_norm: float = 0.3, ctrl_scale: float = 1.0) -> Problem:
    """Generic dense test problem: random Hermitian H0, H_k, Gaussian control samples.

    ``g_norm`` sets dt so that ||H0||_2 * dt ~ g_norm.
    """
    rng = np.random.default_rng(seed)
    H0 = gue(rng, d, 1.0)
    Hk = np.stack([gue(rng, d, 0.5) for _ in range(K)]) if K else np.zeros((0, d, d), np.complex128)
    c = ctrl_scale * rng.standard_normal((K, n_samples(n_steps, integrator)))
    return Problem(f"random_d{d}_K{K}_N{n_steps}_{integrator}", H0, Hk, c, g_norm, integrator, n_steps)


# --- the five benchmark workloads ---------------------------------------------------------


def rabi_qubit(n_steps: int = 1 << 14, T: float = 1000.0) -> Problem:
    """Driven two-level system: H0 = (w0/2) sz, H1 = sx, c(t) = Omega cos(w0 t).

    w0 = 2 pi * 1 GHz, Omega = 2 pi * 10 MHz, T = 1 us, midpoint samples.
    """
    w0 = TWO_PI * 1.0
    Om = TWO_PI * 0.01
    dt = T / n_steps
    t = sample_times(n_steps, dt, "midpoint")
    c = (Om * np.cos(w0 * t))[None, :]
    return Problem("rabi_qubit_d2", 0.5 * w0 * SZ, SX[None].copy(), c, dt, "midpoint", n_steps,
                   meta={"w0": w0, "Omega": Om, "T": T})


def coupled_spins(n_steps: int = 1 << 20, dt: float = 0.01, integrator: str = "magnus4_gl2",
                  n_spins: int = 4) -> Problem:
    """Four coupled spin-1/2 (d = 16): Zeeman + nearest-neighbour ZZ, 8 controls (sx_i, sy_i).

    w_i = 2 pi U[0.5, 1.5] GHz, J_i = U[1, 10] MHz (term 2 pi J/4 sz_i sz_{i+1});
    c_k(t) = sum of 3 sinusoids, frequencies at the spin's carrier +-5 %,
    amplitudes U[0, 2 pi 10 MHz], phases U[0, 2 pi).  dt = 10 ps.
    """
    rng = np.random.default_rng(SEED_BASE + 2)
    w = TWO_PI * rng.uniform(0.5, 1.5, n_spins)
    J = rng.uniform(1e-3, 10e-3, n_spins - 1)
    d = 2 ** n_spins
    H0 = np.zeros((d, d), np.complex128)
    for i in range(n_spins):
        H0 += 0.5 * w[i] * embed(SZ, i, n_spins)
    for i in range(n_spins - 1):
        H0 += (TWO_PI * J[i] / 4.0) * embed(SZ, i, n_spins) @ embed(SZ, i + 1, n_spins)
    Hk = []
    for i in range(n_spins):
        Hk.append(embed(SX, i, n_spins))
        Hk.append(embed(SY, i, n_spins))
    Hk = np.stack(Hk)
    K = Hk.shape[0]
    t = sample_times(n_steps, dt, integrator)
    c = np.zeros((K, t.size))
    for k in range(K):
        f0 = w[k // 2] / TWO_PI
        for _ in range(3):
            f = f0 * (1.0 + rng.uniform(-0.05, 0.05))
            A = rng.uniform(0.0, TWO_PI * 0.01)
            ph = rng.uniform(0.0, TWO_PI)
            c[k] += A * np.sin(TWO_PI * f * t + ph)
    return Problem("coupled_spins_d16", H0, Hk, c, dt, integrator, n_steps,
                   meta={"w": w.tolist(), "J": J.tolist()})


def batched_instances(n_inst: int = 256, dims=(2, 4, 8, 16, 32, 64), seed_offset: int = 3,
                      n_min: float = 1e3, n_max: float = 1e5) -> list[Problem]:
    """Batched sweep: d uniform in ``dims``, N log-uniform in [1e3, 1e5], K uniform in 2..6.

    H0 GUE with ||H0||_2 = 2 pi * 1 GHz, H_k GUE with ||H_k||_2 = 1, piecewise-constant
    Gaussian amplitudes with sigma = 2 pi * 20 MHz, dt = 0.2 / (2 pi * 1 GHz).
    """
    rng = np.random.default_rng(SEED_BASE + seed_offset)
    out = []
    dt = 0.2 / (TWO_PI * 1.0)
    for i in range(n_inst):
        d = int(rng.choice(dims))
        N = int(round(10.0 ** rng.uniform(math.log10(n_min), math.log10(n_max))))
        K = int(rng.integers(2, 7))
        H0 = gue(rng, d, TWO_PI * 1.0)
        Hk = np.stack([gue(rng, d, 1.0) for _ in range(K)])
        c = rng.normal(0.0, TWO_PI * 0.02, (K, N))
        out.append(Problem(f"inst{i}_d{d}_N{N}_K{K}", H0, Hk, c, dt, "midpoint", N))
    return out


def gradient_qubits(n_steps: int = 65536, dt: float = 1.0, n_qubits: int = 3) -> Problem:
    """Optimal-control gradient workload: d = 8, 6 controls, piecewise-constant N(0, (2 pi 20 MHz)^2).

    Rotating-frame H0 = sum_i (delta_i/2) sz_i + sum_i (2 pi J_i / 4) sz_i sz_{i+1},
    delta_i = 2 pi U[-5, 5] MHz, J_i = U[1, 10] MHz; target V Haar-random.  dt = 1 ns.
    """
    rng = np.random.default_rng(SEED_BASE + 4)
    d = 2 ** n_qubits
    delta = TWO_PI * rng.uniform(-5e-3, 5e-3, n_qubits)
    J = rng.uniform(1e-3, 10e-3, n_qubits - 1)
    H0 = np.zeros((d, d), np.complex128)
    for i in range(n_qubits):
        H0 += 0.5 * delta[i] * embed(SZ, i, n_qubits)
    for i in range(n_qubits - 1):
        H0 += (TWO_PI * J[i] / 4.0) * embed(SZ, i, n_qubits) @ embed(SZ, i + 1, n_qubits)
    Hk = []
    for i in range(n_qubits):
        Hk.append(embed(SX, i, n_qubits))
        Hk.append(embed(SY, i, n_qubits))
    Hk = np.stack(Hk)
    c = rng.normal(0.0, TWO_PI * 0.02, (Hk.shape[0], n_steps))
    V = haar_unitary(rng, d)
    return Problem("gradient_qubits_d8", H0, Hk, c, dt, "midpoint", n_steps, V=V)


def dense_stress(n_steps: int = 1 << 16, d: int = 128, K: int = 4, integrator: str = "magnus4_gl2") -> Problem:
    """Dense precision stress: d = 128 GUE H0 (||H0||_2 = 2 pi 100 MHz), 4 GUE controls (||H_k||_2 = 1),
    c_k(t) = sum of 8 Fourier modes a_m sin(2 pi m t / T + phi_m), a_m ~ N(0, (2 pi 10 MHz)^2).
    dt = 0.2 / (2 pi 100 MHz).
    """
    rng = np.random.default_rng(SEED_BASE + 5)
    H0 = gue(rng, d, TWO_PI * 0.1)
    Hk = np.stack([gue(rng, d, 1.0) for _ in range(K)])
    dt = 0.2 / (TWO_PI * 0.1)
    T = n_steps * dt
    t = sample_times(n_steps, dt, integrator)
    c = np.zeros((K, t.size))
    for k in range(K):
        for m in range(1, 9):
            a = rng.normal(0.0, TWO_PI * 0.01)
            ph = rng.uniform(0.0, TWO_PI)
            c[k] += a * np.sin(TWO_PI * m * t / T + ph)
    return Problem(f"dense_stress_d{d}", H0, Hk, c, dt, integrator, n_steps)


def circular_drive(n_steps: int, integrator: str, w0: float = 1.0, w1: float = 0.1, wrf: float = 1.0,
                   t_final: float = 6.0) -> Problem:
    """Qubit under a circularly polarised drive (the paper's convergence example, Sec. 5):
    H(t) = (w0/2) sz + cos(wrf t)(w1/2) sx + sin(wrf t)(w1/2) sy, two controls sx, sy.
    """
    dt = t_final / n_steps
    t = sample_times(n_steps, dt, integrator)
    c = np.stack([0.5 * w1 * np.cos(wrf * t), 0.5 * w1 * np.sin(wrf * t)])
    return Problem(f"circular_drive_{integrator}_N{n_steps}", 0.5 * w0 * SZ, np.stack([SX, SY]), c, dt,
                   integrator, n_steps, meta={"w0": w0, "w1": w1, "wrf": wrf, "t": t_final})
