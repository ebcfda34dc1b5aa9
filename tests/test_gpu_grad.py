"""Adjoint gradient on the GPU against the oracle's Daleckii-Krein gradient and finite differences
(midpoint rule and both fourth-order Magnus integrators).

FP64: the adjoint gradient agrees with the oracle to 1e-9 relative to max |g|
(the two use different exponential and Frechet-derivative algorithms; the bound
leaves room for N accumulated rounding errors of ~1e-15), and with central
finite differences of the GPU forward (h = 1e-6) to 1e-6 relative, as the
optimal-control workload requires.  FP32: relative to max |g|, the gradient's error grows like
the forward FP32 error (a random walk of slice rounding, u sqrt(N)); the bound GRAD32_REL is a
few times the measured error (4.8e-5 at N = 65 536 with exact inputs).
"""

import math

import numpy as np
import pytest

import oracle
from paper_2108_07126_gb300 import workloads as wl
from tolerances import check

pytestmark = pytest.mark.gpu

GRAD32_REL = 2e-4  # FP32 gradient vs the oracle, relative to max |g|


@pytest.fixture()
def prop():
    import torch

    from paper_2108_07126_gb300.binding import Propagator

    assert torch.cuda.is_available()
    p = Propagator(0)
    yield p
    p.close()


def gpu_grad(prop, prob, V, prec="fp64", subchunk=0, integrator="midpoint"):
    import torch

    from paper_2108_07126_gb300 import binding as b

    cdt = torch.complex128 if prec == "fp64" else torch.complex64
    rdt = torch.float64 if prec == "fp64" else torch.float32
    prop.set_option(b.PARAMENT_OPT_GRAD_SUBCHUNK, subchunk)
    prop.set_hamiltonians(torch.as_tensor(prob.H0).to(cdt), torch.as_tensor(prob.Hk).to(cdt), integrator)
    prop.set_controls(torch.as_tensor(prob.c).to(rdt), prob.dt, prob.n_steps)
    loss, grad, U = prop.propagate_grad(torch.as_tensor(V).to(cdt), prec, want_U=True)
    torch.cuda.synchronize()
    return loss, grad.cpu().numpy().astype(np.float64), U.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("d,K,N", [(2, 1, 1), (2, 2, 7), (3, 2, 300), (4, 3, 129), (8, 6, 1000), (5, 4, 64),
                                   (16, 3, 257), (12, 2, 77)])
def test_fp64_gradient_matches_oracle(prop, d, K, N):
    prob = wl.random_problem(d, K, N, "midpoint", seed=500 + d * 10 + K, g_norm=0.4)
    V = wl.haar_unitary(np.random.default_rng(d + N), d)
    loss, grad, U = gpu_grad(prop, prob, V)
    l_ref, g_ref, U_ref = oracle.loss_and_gradient(prob.H0, prob.Hk, prob.c, prob.dt, V)
    assert abs(loss - l_ref) <= 1e-11
    assert np.max(np.abs(U - U_ref)) <= 1e-11
    assert np.max(np.abs(grad - g_ref)) <= 1e-9 * np.max(np.abs(g_ref))


@pytest.mark.parametrize("subchunk", [1, 3, 7, 50])
def test_checkpointed_sweeps_agree(prop, subchunk):
    prob = wl.random_problem(4, 2, 2000, "midpoint", seed=77, g_norm=0.3)
    V = wl.haar_unitary(np.random.default_rng(3), 4)
    _, g_full, _ = gpu_grad(prop, prob, V)
    _, g_ck, _ = gpu_grad(prop, prob, V, subchunk=subchunk)
    assert prop.stats()["grad_subchunk"] == subchunk
    assert np.max(np.abs(g_ck - g_full)) <= 1e-12 * np.max(np.abs(g_full))


def test_gradient_workload_full_size(prop):
    """Three qubits, 6 controls, N = 65536: adjoint vs oracle (full) and vs central FD (subset)."""
    import torch

    from paper_2108_07126_gb300 import binding as b

    prob = wl.gradient_qubits()
    loss, grad, U = gpu_grad(prop, prob, prob.V)
    l_ref, g_ref, U_ref = oracle.loss_and_gradient(prob.H0, prob.Hk, prob.c, prob.dt, prob.V)
    assert abs(loss - l_ref) <= 1e-10
    assert np.max(np.abs(grad - g_ref)) <= 1e-9 * np.max(np.abs(g_ref))
    # central finite differences of the GPU FP64 forward, h = 1e-6 (rad/ns)
    rng = np.random.default_rng(11)
    entries = [(int(rng.integers(0, 6)), int(rng.integers(0, prob.n_steps))) for _ in range(12)]
    H0 = torch.as_tensor(prob.H0).cuda()
    Hk = torch.as_tensor(prob.Hk).cuda()
    prop.set_hamiltonians(H0, Hk, "midpoint")
    Vh = prob.V.conj().T

    def loss_of(c):
        prop.set_controls(torch.as_tensor(c).cuda(), prob.dt, prob.n_steps)
        Um = prop.propagate("fp64").cpu().numpy()
        return 1.0 - abs(np.trace(Vh @ Um)) ** 2 / 64.0

    fd = []
    for (k, j) in entries:
        cp = prob.c.copy()
        cm = prob.c.copy()
        cp[k, j] += 1e-6
        cm[k, j] -= 1e-6
        fd.append((loss_of(cp) - loss_of(cm)) / 2e-6)
    fd = np.array(fd)
    ga = np.array([grad[k, j] for (k, j) in entries])
    assert np.max(np.abs(ga - fd)) <= 1e-6 * np.max(np.abs(fd))


def test_fp32_gradient_error(prop):
    prob = wl.gradient_qubits(n_steps=8192)
    loss, grad, U = gpu_grad(prop, prob, prob.V, "fp32")
    l_ref, g_ref, _ = oracle.loss_and_gradient(prob.H0, prob.Hk, prob.c, prob.dt, prob.V)
    rel = np.max(np.abs(grad - g_ref)) / np.max(np.abs(g_ref))
    check(rel, GRAD32_REL, "fp32 gradient, relative")
    check(abs(loss - l_ref), 4e-6, "fp32 loss")


def test_gradient_invariants(prop):
    d = 4
    prob = wl.random_problem(d, 2, 50, "midpoint", seed=90, g_norm=0.4)
    rng = np.random.default_rng(91)
    Hk = np.concatenate([prob.Hk, np.eye(d, dtype=np.complex128)[None]])
    c = np.concatenate([prob.c, rng.standard_normal((1, 50))])
    prob2 = wl.Problem("with_identity", prob.H0, Hk, c, prob.dt, "midpoint", 50)
    V = wl.haar_unitary(rng, d)
    loss, grad, U = gpu_grad(prop, prob2, V)
    assert np.max(np.abs(grad[-1])) <= 1e-12  # global phase does not change L
    loss_u, grad_u, _ = gpu_grad(prop, prob2, U)
    assert abs(loss_u) <= 1e-12 and np.max(np.abs(grad_u)) <= 1e-10


@pytest.mark.parametrize("integrator", ["magnus4_gl2", "magnus4_simpson"])
@pytest.mark.parametrize("d,K,N", [(2, 1, 1), (2, 2, 9), (3, 3, 200), (4, 2, 129), (8, 4, 300), (16, 3, 65),
                                   (5, 5, 31)])
def test_fp64_magnus_gradient_matches_oracle(prop, integrator, d, K, N):
    """Magnus integrators: every sample's derivative through the effective-control basis
    (commutator terms included; Simpson end samples get the contributions of both slices)."""
    prob = wl.random_problem(d, K, N, integrator, seed=540 + d * 10 + K, g_norm=0.4)
    V = wl.haar_unitary(np.random.default_rng(d + N + 1), d)
    loss, grad, U = gpu_grad(prop, prob, V, integrator=integrator)
    l_ref, g_ref, U_ref = oracle.loss_and_gradient(prob.H0, prob.Hk, prob.c, prob.dt, V, integrator)
    assert grad.shape == g_ref.shape == prob.c.shape
    assert abs(loss - l_ref) <= 1e-11
    assert np.max(np.abs(U - U_ref)) <= 1e-11
    assert np.max(np.abs(grad - g_ref)) <= 1e-9 * np.max(np.abs(g_ref))


@pytest.mark.parametrize("integrator", ["magnus4_gl2", "magnus4_simpson"])
def test_fp32_magnus_gradient_error(prop, integrator):
    prob = wl.random_problem(8, 3, 2000, integrator, seed=560, g_norm=0.3)
    V = wl.haar_unitary(np.random.default_rng(561), 8)
    loss, grad, _ = gpu_grad(prop, prob, V, "fp32", integrator=integrator)
    l_ref, g_ref, _ = oracle.loss_and_gradient(prob.H0, prob.Hk, prob.c, prob.dt, V, integrator)
    rel = np.max(np.abs(grad - g_ref)) / np.max(np.abs(g_ref))
    check(rel, GRAD32_REL, ("fp32 Magnus gradient, relative", integrator))


def test_magnus_gradient_checkpoints_agree(prop):
    prob = wl.random_problem(4, 2, 700, "magnus4_simpson", seed=570, g_norm=0.3)
    V = wl.haar_unitary(np.random.default_rng(571), 4)
    _, g_full, _ = gpu_grad(prop, prob, V, integrator="magnus4_simpson")
    _, g_ck, _ = gpu_grad(prop, prob, V, subchunk=5, integrator="magnus4_simpson")
    assert np.max(np.abs(g_ck - g_full)) <= 1e-12 * np.max(np.abs(g_full))


def test_gradient_errors(prop):
    import torch

    from paper_2108_07126_gb300 import binding as b

    prob = wl.random_problem(32, 1, 10, "midpoint", seed=1)
    prop.set_hamiltonians(torch.as_tensor(prob.H0), torch.as_tensor(prob.Hk), "midpoint")
    prop.set_controls(torch.as_tensor(prob.c), prob.dt, 10)
    with pytest.raises(b.ParamentError) as e:
        prop.propagate_grad(np.eye(32), "fp32_tc_tf32x3")
    assert e.value.status == b.PARAMENT_ERR_UNSUPPORTED


# --- d > 16: one thread block per leaf, block-level adjoint -------------------------------------


@pytest.mark.parametrize("integrator", ["midpoint", "magnus4_gl2", "magnus4_simpson"])
@pytest.mark.parametrize("d,K,N", [(17, 2, 45), (32, 2, 40), (64, 2, 21), (100, 1, 9), (128, 2, 7), (200, 1, 4)])
def test_large_d_fp64_gradient_matches_oracle(prop, integrator, d, K, N):
    """FP64 adjoint gradient for d > 16 against the oracle's Daleckii-Krein gradient (all three
    integrators), with the loss and U(T) from the FP64 leaf scans."""
    if d >= 100 and integrator != "magnus4_gl2":
        pytest.skip("the largest sizes run one integrator (FP64 products at d = 128..256 are slow)")
    prob = wl.random_problem(d, K, N, integrator, seed=580 + d + K, g_norm=0.4)
    V = wl.haar_unitary(np.random.default_rng(d + N + 7), d)
    loss, grad, U = gpu_grad(prop, prob, V, integrator=integrator)
    l_ref, g_ref, U_ref = oracle.loss_and_gradient(prob.H0, prob.Hk, prob.c, prob.dt, V, integrator)
    assert grad.shape == g_ref.shape == prob.c.shape
    assert abs(loss - l_ref) <= 1e-11
    assert np.max(np.abs(U - U_ref)) <= 1e-11
    assert np.max(np.abs(grad - g_ref)) <= 1e-9 * np.max(np.abs(g_ref))


def test_large_d_gradient_checkpoints_agree(prop):
    """Leaves longer than the sub-chunk buffer re-compute their prefixes from checkpoints: the same
    gradient as with the whole leaf in the buffer."""
    prob = wl.random_problem(40, 2, 700, "magnus4_gl2", seed=590, g_norm=0.3)
    V = wl.haar_unitary(np.random.default_rng(591), 40)
    _, g_full, _ = gpu_grad(prop, prob, V, integrator="magnus4_gl2")
    _, g_ck, _ = gpu_grad(prop, prob, V, subchunk=2, integrator="magnus4_gl2")
    assert prop.stats()["grad_subchunk"] == 2
    assert np.max(np.abs(g_full - g_ck)) <= 1e-12 * np.max(np.abs(g_full))


def test_large_d_fp32_gradient(prop):
    prob = wl.random_problem(64, 3, 300, "magnus4_gl2", seed=592, g_norm=0.3)
    V = wl.haar_unitary(np.random.default_rng(593), 64)
    loss, grad, _ = gpu_grad(prop, prob, V, "fp32", integrator="magnus4_gl2")
    l_ref, g_ref, _ = oracle.loss_and_gradient(prob.H0, prob.Hk, prob.c, prob.dt, V, "magnus4_gl2")
    check(np.max(np.abs(grad - g_ref)) / np.max(np.abs(g_ref)), GRAD32_REL, "fp32 gradient d = 64, relative")
    check(abs(loss - l_ref), 4e-6, "fp32 loss d = 64")


def test_autograd_function(prop):
    import torch

    from paper_2108_07126_gb300.autograd import gate_infidelity

    prob = wl.random_problem(3, 2, 40, "midpoint", seed=92, g_norm=0.3)
    V = wl.haar_unitary(np.random.default_rng(5), 3)
    prop.set_hamiltonians(torch.as_tensor(prob.H0), torch.as_tensor(prob.Hk), "midpoint")
    c = torch.as_tensor(prob.c).cuda().requires_grad_(True)
    L = gate_infidelity(prop, c, V, prob.dt)
    (g,) = torch.autograd.grad(3.0 * L, c)
    l_ref, g_ref, _ = oracle.loss_and_gradient(prob.H0, prob.Hk, prob.c, prob.dt, V)
    assert abs(L.item() - l_ref) <= 1e-11
    assert np.max(np.abs(g.cpu().numpy() - 3.0 * g_ref)) <= 1e-9 * 3.0 * np.max(np.abs(g_ref))


@pytest.mark.parametrize("integrator", ["midpoint", "magnus4_simpson"])
def test_gradient_with_pinned_host_controls(prop, integrator):
    """Controls in page-locked host memory (read by the kernels in place) give bit-for-bit the
    loss and gradient of device-resident controls."""
    import torch

    from paper_2108_07126_gb300 import binding as b

    prob = wl.random_problem(4, 2, 700, integrator, seed=5150, g_norm=0.3)
    V = wl.haar_unitary(np.random.default_rng(5151), 4)
    prop.set_hamiltonians(torch.as_tensor(prob.H0), torch.as_tensor(prob.Hk), integrator)
    c = torch.as_tensor(prob.c)
    prop.set_controls(c.cuda(), prob.dt, prob.n_steps)
    loss_d, g_d = prop.propagate_grad(V, "fp64")
    pinned = c.pin_memory()
    b.parament_set_controls(prop.ctx, pinned.data_ptr(), b.PARAMENT_F64, prob.n_steps, prob.dt)
    loss_h, g_h = prop.propagate_grad(V, "fp64")
    torch.cuda.synchronize()
    assert loss_h == loss_d and torch.equal(g_h, g_d)
