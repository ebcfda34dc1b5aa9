"""FP64 CPU oracle for slice-wise propagation (Herb & Welter, "Parallel time
integration using Batched BLAS routines", arXiv 2108.07126).

TEST INFRASTRUCTURE ONLY.  This module is the slow, plain reference that the
CUDA library is checked against.  Only the test suite, the smoke check and the
CPU-baseline leg of the benchmark may import it; the product path never does.
It shares no code with the CUDA library (no kernels, headers, tables or
helpers); the only thing both sides see is the seeded input arrays.

What it computes, each piece following the paper's definitions:

* ``hamiltonian``        -- H(t) = H0 + sum_k c_k(t) H_k          (Sec. 2, Eq. format_control)
* ``slice_exponents``    -- the Hermitian exponent G_j of every slice, so that
                            U_j = exp(-i G_j):
    - midpoint rule      G_j = dt * H(t_j + dt/2)                 (Sec. 3.2 and Sec. 4: Omega_1 by the mid-point rule)
    - Gauss-Legendre 4   G_j = dt/2 (H1 + H2) + i sqrt(3) dt^2/12 [H1, H2]
                         with H1, H2 at t_j + dt (1/2 -+ sqrt(3)/6)   (Sec. 4, Eq. magnus: Omega_1 + Omega_2)
    - Simpson 4          G_j = dt/6 (H1 + 4 H2 + H3) + i dt^2/12 [H1, H3]
                         with H1, H2, H3 at t_j, t_j + dt/2, t_j + dt  (Sec. 4, the Simpson/trapezoid exponent)
  The sign of the commutator term follows from Omega_2 = -1/2 int int [H(t1), H(t2)]
  (Sec. 4, Eq. magnus); the paper's printed Simpson exponent carries the
  opposite sign, which gives a second-order method (see the pins).
* ``exact_slice_propagators`` -- U_j = exp(-i G_j) exactly (up to rounding),
  by a Hermitian eigendecomposition G = Q diag(lam) Q^dagger, so
  U_j = Q diag(exp(-i lam)) Q^dagger.  (Sec. 2.1 names decomposition methods as
  the natural choice for Hermitian matrices; the CUDA path uses a series
  instead, so the two agree only up to rounding.)
* ``ordered_product``    -- U(T) = U_N ... U_1 (Sec. 2, Eq. slices: later slices
  on the left) evaluated by the pairwise tree of Sec. 2.2: consecutive pairs
  are multiplied, the number of matrices halves each round, an odd leftover
  (the latest slice) is carried to the next round unchanged.
* ``trajectory``         -- the propagator at intermediate times, U(t_n) = U_n ... U_1
  for n = every, 2 every, ... and the last slice N (Sec. 2, Eq. slices read at
  t_n instead of T), or the states psi(t_n) = U(t_n) psi_0 (Sec. 2, the state
  form of the Schroedinger equation); a plain sequential left-multiplication
  in time order.
* ``loss_and_gradient``  -- gate-fidelity loss L = 1 - |Tr(V^dagger U)|^2 / d^2 and
  dL/dc_k(s) for every control sample and every integrator (chain rule through
  the exponent formulas, ``exponent_derivatives``), with the Frechet derivative
  of exp taken from the Daleckii-Krein formula (Sec. 7 motivates the gradient
  for GRAPE; the paper itself gives no gradient formula).

All arithmetic is complex128 / float64.  Parity is pinned by the tests in
``tests/test_oracle_pins.py`` (closed forms, convergence orders, brute-force
ODE integration, finite differences); no function here is "parity unpinned".
"""

from __future__ import annotations

import math

import numpy as np

MIDPOINT = "midpoint"
MAGNUS4_GL2 = "magnus4_gl2"
MAGNUS4_SIMPSON = "magnus4_simpson"
INTEGRATORS = (MIDPOINT, MAGNUS4_GL2, MAGNUS4_SIMPSON)


def samples_per_run(n_steps: int, integrator: str) -> int:
    """Number S of control samples per control for ``n_steps`` slices.

    Midpoint: one sample per slice at its centre (S = N).  Gauss-Legendre:
    two node samples per slice (S = 2N).  Simpson: both end points and the
    centre of every slice, end points shared with the neighbours (S = 2N + 1).
    """
    if integrator == MIDPOINT:
        return n_steps
    if integrator == MAGNUS4_GL2:
        return 2 * n_steps
    if integrator == MAGNUS4_SIMPSON:
        return 2 * n_steps + 1
    raise ValueError(f"unknown integrator {integrator!r}")


def hamiltonian(H0: np.ndarray, Hk: np.ndarray, c: np.ndarray) -> np.ndarray:
    """H = H0 + sum_k c_k H_k  (Sec. 2, Eq. format_control).

    ``H0`` is (d, d), ``Hk`` is (K, d, d), ``c`` is (K,) or (K, M) for M time
    points; the result is (d, d) or (M, d, d).
    """
    H0 = np.asarray(H0, dtype=np.complex128)
    Hk = np.asarray(Hk, dtype=np.complex128).reshape(-1, H0.shape[0], H0.shape[0])
    c = np.asarray(c, dtype=np.float64)
    if c.ndim == 1:
        return H0 + np.einsum("k,kab->ab", c, Hk)
    return H0[None] + np.einsum("km,kab->mab", c, Hk)


def commutator(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """[A, B] = AB - BA, batched over leading axes (Sec. 4)."""
    return A @ B - B @ A


def slice_exponents(H0, Hk, c, dt: float, integrator: str) -> np.ndarray:
    """Hermitian exponents G_j (N, d, d) with U_j = exp(-i G_j).

    ``c`` is the (K, S) array of real control samples, S as in
    ``samples_per_run``; ``dt`` is the slice duration.
    """
    c = np.asarray(c, dtype=np.float64)
    K = np.asarray(Hk).reshape(-1, np.asarray(H0).shape[0], np.asarray(H0).shape[0]).shape[0]
    c = c.reshape(K, -1)
    S = c.shape[1]
    if integrator == MIDPOINT:
        # Omega_1 by the mid-point rule: the Hamiltonian at the slice centre.
        return dt * hamiltonian(H0, Hk, c)
    if integrator == MAGNUS4_GL2:
        if S % 2:
            raise ValueError("Gauss-Legendre needs two samples per slice")
        H1 = hamiltonian(H0, Hk, c[:, 0::2])  # node t_j + dt (1/2 - sqrt(3)/6)
        H2 = hamiltonian(H0, Hk, c[:, 1::2])  # node t_j + dt (1/2 + sqrt(3)/6)
        # Omega_1: two-node Gauss-Legendre quadrature of the Hamiltonian.
        # Omega_2: the double integral of [H(t1), H(t2)] on the same nodes;
        # Omega = -i G  gives the +i sign in front of [H1, H2].
        return 0.5 * dt * (H1 + H2) + 1j * (math.sqrt(3.0) * dt * dt / 12.0) * commutator(H1, H2)
    if integrator == MAGNUS4_SIMPSON:
        if S % 2 != 1 or S < 1:
            raise ValueError("Simpson needs 2N + 1 samples")
        H1 = hamiltonian(H0, Hk, c[:, 0:S - 1:2])   # slice start
        H2 = hamiltonian(H0, Hk, c[:, 1:S:2])       # slice centre
        H3 = hamiltonian(H0, Hk, c[:, 2:S:2])       # slice end
        # Omega_1 by Simpson's rule, Omega_2 by the trapezoidal rule (Sec. 4).
        return (dt / 6.0) * (H1 + 4.0 * H2 + H3) + 1j * (dt * dt / 12.0) * commutator(H1, H3)
    raise ValueError(f"unknown integrator {integrator!r}")


def exact_slice_propagators(G: np.ndarray) -> np.ndarray:
    """U_j = exp(-i G_j) for Hermitian G_j via eigendecomposition."""
    G = np.asarray(G, dtype=np.complex128)
    lam, Q = np.linalg.eigh(G)
    return (Q * np.exp(-1j * lam)[..., None, :]) @ np.conj(np.swapaxes(Q, -1, -2))


def ordered_product(U: np.ndarray) -> np.ndarray:
    """U_N ... U_1 by the pairwise tree of Sec. 2.2.

    ``U`` is (N, d, d) in time order (U[0] is the first slice).  Each round
    multiplies consecutive pairs, the later slice on the left; an odd
    leftover is carried to the next round unchanged.  N = 0 gives the
    identity.
    """
    U = np.asarray(U, dtype=np.complex128)
    if U.shape[0] == 0:
        return np.eye(U.shape[-1], dtype=np.complex128)
    while U.shape[0] > 1:
        n = U.shape[0]
        pairs = U[1:n - n % 2:2] @ U[0:n - n % 2:2]
        U = np.concatenate([pairs, U[n - 1:]]) if n % 2 else pairs
    return U[0]


def propagate(H0, Hk, c, dt: float, integrator: str = MIDPOINT) -> np.ndarray:
    """Full propagator U(T) = U_N ... U_1 (Sec. 2, Eq. slices)."""
    G = slice_exponents(H0, Hk, c, dt, integrator)
    return ordered_product(exact_slice_propagators(G))


def trajectory_times(n_steps: int, every: int) -> np.ndarray:
    """Slice counts n of the outputs: every, 2 every, ..., and n_steps if it is not a multiple."""
    n = np.arange(every, n_steps + 1, every, dtype=np.int64)
    if n_steps % every:
        n = np.append(n, n_steps)
    return n


def trajectory(H0, Hk, c, dt: float, integrator: str = MIDPOINT, every: int = 1, psi0=None) -> np.ndarray:
    """U(t_n) = U_n ... U_1 at n in ``trajectory_times(N, every)`` (Sec. 2, Eq. slices).

    Sequential: R <- U_j R for j = 1..N (later slice on the left), R kept at the
    output slices.  With ``psi0`` (length d) the states psi(t_n) = U(t_n) psi0
    are returned instead, shape (n_out, d); otherwise (n_out, d, d).
    """
    G = slice_exponents(H0, Hk, c, dt, integrator)
    Us = exact_slice_propagators(G)
    N, d = G.shape[0], np.asarray(H0).shape[-1]
    keep = set(int(n) for n in trajectory_times(N, every))
    R = np.eye(d, dtype=np.complex128)
    out = []
    for j in range(N):
        R = Us[j] @ R
        if j + 1 in keep:
            out.append(R.copy())
    out = np.array(out, dtype=np.complex128).reshape(len(out), d, d)
    if psi0 is not None:
        return out @ np.asarray(psi0, dtype=np.complex128)
    return out


def gate_loss(U: np.ndarray, V: np.ndarray) -> float:
    """L = 1 - |Tr(V^dagger U)|^2 / d^2 (gate infidelity)."""
    d = U.shape[-1]
    z = np.trace(np.conj(V).T @ U)
    return float(1.0 - abs(z) ** 2 / d ** 2)


def frechet_phi(lam: np.ndarray) -> np.ndarray:
    """Divided differences of exp(-i x) on the eigenvalues (Daleckii-Krein).

    Phi_ab = (e^{-i l_a} - e^{-i l_b}) / (-i l_a + i l_b), Phi_aa = e^{-i l_a},
    written in the cancellation-free form
    e^{-i (l_a + l_b)/2} * sin(delta) / delta with delta = (l_a - l_b)/2.
    """
    la = lam[..., :, None]
    lb = lam[..., None, :]
    delta = 0.5 * (la - lb)
    return np.exp(-0.5j * (la + lb)) * np.sinc(delta / np.pi)


def frechet_exp(G: np.ndarray, E: np.ndarray) -> np.ndarray:
    """L_X(E): Frechet derivative of exp at X = -i G in direction E.

    Daleckii-Krein: with G = Q diag(lam) Q^dagger,
    L_X(E) = Q [ (Q^dagger E Q) o Phi ] Q^dagger  (o = elementwise product).
    """
    lam, Q = np.linalg.eigh(np.asarray(G, dtype=np.complex128))
    Qh = np.conj(np.swapaxes(Q, -1, -2))
    return Q @ ((Qh @ E @ Q) * frechet_phi(lam)) @ Qh


def exponent_derivatives(H0, Hk, c, dt: float, integrator: str):
    """dG_j / dc_k(s) for every slice j, control k and sample s the slice reads.

    Returns a list of (offset, D) with D of shape (N, K, d, d): D[j, k] is the derivative of
    G_j with respect to the sample at index offset + 2 j (offset + j for the midpoint rule)
    of control k, from the exponent formulas of ``slice_exponents`` (Sec. 4, Eq. magnus):
      midpoint    G = dt H                              dG/dc_k = dt H_k
      GL4         G = dt/2 (H1 + H2) + i w [H1, H2],    w = sqrt(3) dt^2 / 12
                  dG/dc1_k = dt/2 H_k + i w [H_k, H2],  dG/dc2_k = dt/2 H_k + i w [H1, H_k]
      Simpson     G = dt/6 (H1 + 4 H2 + H3) + i (dt^2/12) [H1, H3]
                  dG/dc1_k = dt/6 H_k + i (dt^2/12) [H_k, H3],  dG/dc2_k = 4 dt/6 H_k,
                  dG/dc3_k = dt/6 H_k + i (dt^2/12) [H1, H_k]
    """
    H0 = np.asarray(H0, dtype=np.complex128)
    d = H0.shape[0]
    Hk = np.asarray(Hk, dtype=np.complex128).reshape(-1, d, d)
    K = Hk.shape[0]
    c = np.asarray(c, dtype=np.float64).reshape(K, -1)
    S = c.shape[1]
    if integrator == MIDPOINT:
        N = S
        return [(0, np.broadcast_to(dt * Hk[None], (N, K, d, d)))]
    if integrator == MAGNUS4_GL2:
        N = S // 2
        H1 = hamiltonian(H0, Hk, c[:, 0::2])[:, None]      # (N, 1, d, d)
        H2 = hamiltonian(H0, Hk, c[:, 1::2])[:, None]
        w = math.sqrt(3.0) * dt * dt / 12.0
        Hb = Hk[None]                                       # (1, K, d, d)
        D1 = 0.5 * dt * Hb + 1j * w * commutator(Hb, H2)
        D2 = 0.5 * dt * Hb + 1j * w * commutator(H1, Hb)
        return [(0, D1), (1, D2)]
    if integrator == MAGNUS4_SIMPSON:
        N = (S - 1) // 2
        H1 = hamiltonian(H0, Hk, c[:, 0:S - 1:2])[:, None]
        H3 = hamiltonian(H0, Hk, c[:, 2:S:2])[:, None]
        w = dt * dt / 12.0
        Hb = np.broadcast_to(Hk[None], (N, K, d, d))
        D1 = dt / 6.0 * Hb + 1j * w * commutator(Hk[None], H3)
        D2 = 4.0 * dt / 6.0 * Hb
        D3 = dt / 6.0 * Hb + 1j * w * commutator(H1, Hk[None])
        return [(0, D1), (1, D2), (2, D3)]
    raise ValueError(f"unknown integrator {integrator!r}")


def loss_and_gradient(H0, Hk, c, dt: float, V, integrator: str = MIDPOINT):
    """Loss L, gradient dL/dc (K, S) over the control samples, and U(T).

    U = S_j U_j P_{j-1} with the exclusive prefix P_{j-1} = U_{j-1} ... U_1
    and suffix S_j = U_N ... U_{j+1}; with z = Tr(V^dagger U) and X_j = -i G_j,
    dz/dc = sum_j Tr(Lambda_j L_{X_j}(dX_j/dc)), Lambda_j = P_{j-1} V^dagger S_j,
    dX_j/dc = -i dG_j/dc (``exponent_derivatives``: one sample enters one slice, or two
    neighbouring slices for the shared Simpson end points), and
    dL/dc = -(2/d^2) Re(conj(z) dz/dc).
    """
    H0 = np.asarray(H0, dtype=np.complex128)
    d = H0.shape[0]
    Hk = np.asarray(Hk, dtype=np.complex128).reshape(-1, d, d)
    K = Hk.shape[0]
    c = np.asarray(c, dtype=np.float64).reshape(K, -1)
    V = np.asarray(V, dtype=np.complex128)

    G = slice_exponents(H0, Hk, c, dt, integrator)
    N = G.shape[0]
    lam, Q = np.linalg.eigh(G)
    Qh = np.conj(np.swapaxes(Q, -1, -2))
    Uj = (Q * np.exp(-1j * lam)[:, None, :]) @ Qh

    # exclusive prefixes P_{j-1} and suffixes S_j by their definitions
    P = np.empty_like(Uj)
    S = np.empty_like(Uj)
    acc = np.eye(d, dtype=np.complex128)
    for j in range(N):
        P[j] = acc
        acc = Uj[j] @ acc
    U = acc
    acc = np.eye(d, dtype=np.complex128)
    for j in range(N - 1, -1, -1):
        S[j] = acc
        acc = acc @ Uj[j]

    z = np.trace(np.conj(V).T @ U)
    loss = float(1.0 - abs(z) ** 2 / d ** 2)
    Lam = P @ np.conj(V).T @ S                       # (N, d, d)
    # Tr(Lam L_X(E)) = sum_ab (Q^dag Lam Q)_ba (Q^dag E Q)_ab Phi_ab
    Lt = Qh @ Lam @ Q                                # (N, d, d)
    phi = frechet_phi(lam)                           # (N, d, d)
    dz = np.zeros(c.shape, dtype=np.complex128)      # (K, S)
    step = 1 if integrator == MIDPOINT else 2
    for off, Dg in exponent_derivatives(H0, Hk, c, dt, integrator):
        E = -1j * np.asarray(Dg)                     # (N, K, d, d)
        Et = np.einsum("nab,nkbc,ncd->nkad", Qh, E, Q)
        dzr = np.einsum("nba,nkab,nab->kn", Lt, Et, phi)  # (K, N)
        for j in range(N):
            dz[:, off + step * j] += dzr[:, j]
    grad = -(2.0 / d ** 2) * np.real(np.conj(z) * dz)
    return loss, grad, U


def effective_control_count(n_ctrl: int) -> int:
    """Number of effective controls of the fourth-order Magnus exponent.

    The exponent is a real combination of H_k, i[H_0, H_k] and i[H_k, H_k']
    for k < k': K + K + K(K-1)/2 = 3K/2 + K^2/2 (Sec. 4, Eq. magnus_coeffs).
    """
    return n_ctrl + n_ctrl + n_ctrl * (n_ctrl - 1) // 2
