"""parament_propagate_noalloc against the context entry point, through the C ABI.

The no-allocation entry point is for callers that cannot allocate device
memory (an application that owns all device memory through its own
allocator, or a latency-critical loop that cannot afford the synchronisation
of cudaMalloc / cudaFree); it keeps its intermediates in one static device
array.  Each case calls it twice in a row -- the array keeps the previous
call's contents, so the second call checks that the state a call needs is
cleared -- and compares both results with parament_propagate on the same
inputs, within the parity tolerances of the other GPU tests (1e-11 in FP64,
20 u d sqrt(N) in FP32).

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""

import math

import numpy as np
import pytest

from paper_2108_07126_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL64 = 1e-11
U32 = 2.0 ** -24


def tol32(d, n):
    return 20.0 * U32 * max(d, 2) * math.sqrt(max(n, 1)) + 1e-6


CASES = [
    ("coupled_spins", lambda: wl.coupled_spins(n_steps=1 << 14), "fp64"),
    ("coupled_spins", lambda: wl.coupled_spins(n_steps=1 << 14), "fp32"),
    ("random_d5_midpoint", lambda: wl.random_problem(5, 3, 3001, "midpoint", seed=41, g_norm=0.5), "fp64"),
    ("random_d3_simpson", lambda: wl.random_problem(3, 2, 777, "magnus4_simpson", seed=42, g_norm=0.3), "fp32"),
    ("rabi_qubit", lambda: wl.rabi_qubit(), "fp64"),
]


@pytest.mark.parametrize("name,make,prec", CASES, ids=[f"{c[0]}-{c[2]}" for c in CASES])
def test_noalloc_matches_context_entry_point(name, make, prec):
    import torch

    from paper_2108_07126_gb300 import binding as b

    assert torch.cuda.is_available()
    prob = make()
    cdt = torch.complex128 if prec == "fp64" else torch.complex64
    rdt = torch.float64 if prec == "fp64" else torch.float32
    H0 = torch.as_tensor(prob.H0).to(cdt).cuda().contiguous()
    Hk = torch.as_tensor(prob.Hk).to(cdt).cuda().contiguous()
    c = torch.as_tensor(prob.c).to(rdt).cuda().contiguous()
    d, K = prob.dim, prob.n_ctrl
    dtype = b.PARAMENT_C128 if prec == "fp64" else b.PARAMENT_C64
    cdtype = b.PARAMENT_F64 if prec == "fp64" else b.PARAMENT_F32
    p = b.PRECISIONS[prec]
    integ = b.INTEGRATORS[prob.integrator]

    # the existing entry point
    ctx = b.parament_create(0, None)
    try:
        b.parament_set_hamiltonians(ctx, d, K, H0.data_ptr(), Hk.data_ptr(), dtype, integ)
        b.parament_set_controls(ctx, c.data_ptr(), cdtype, prob.n_steps, prob.dt)
        U_ref = torch.empty(d, d, dtype=cdt, device="cuda")
        b.parament_propagate(ctx, U_ref.data_ptr(), p)
        torch.cuda.synchronize()
    finally:
        b.parament_destroy(ctx)
    U_ref = U_ref.cpu().numpy().astype(np.complex128)

    tol = TOL64 if prec == "fp64" else tol32(d, prob.n_steps)
    for call in range(2):
        U = torch.full((d, d), float("nan"), dtype=cdt, device="cuda")
        st = b.raw_call("parament_propagate_noalloc", d, K, H0.data_ptr(), Hk.data_ptr(), dtype, integ,
                        c.data_ptr(), cdtype, prob.n_steps, prob.dt, U.data_ptr(), p, None)
        assert st == b.PARAMENT_OK, b.parament_status_string(st)
        torch.cuda.synchronize()
        U = U.cpu().numpy().astype(np.complex128)
        err = np.max(np.abs(U - U_ref))
        assert err <= tol, (name, prec, call, err)


def test_noalloc_rejects_what_it_cannot_hold():
    import torch

    from paper_2108_07126_gb300 import binding as b

    H = torch.eye(32, dtype=torch.complex128, device="cuda")
    U = torch.empty(32, 32, dtype=torch.complex128, device="cuda")
    st = b.raw_call("parament_propagate_noalloc", 32, 0, H.data_ptr(), None, b.PARAMENT_C128, b.PARAMENT_MIDPOINT,
                    None, b.PARAMENT_F64, 4, 0.1, U.data_ptr(), b.PARAMENT_PREC_FP64, None)
    assert st == b.PARAMENT_ERR_INVALID_VALUE
    # nine controls with a Magnus integrator need 1 + 9 * 12 / 2 = 55 > 45 basis matrices
    H = torch.eye(2, dtype=torch.complex128, device="cuda")
    Hk = torch.zeros(9, 2, 2, dtype=torch.complex128, device="cuda")
    c = torch.zeros(9, 8, dtype=torch.float64, device="cuda")
    U = torch.empty(2, 2, dtype=torch.complex128, device="cuda")
    st = b.raw_call("parament_propagate_noalloc", 2, 9, H.data_ptr(), Hk.data_ptr(), b.PARAMENT_C128,
                    b.PARAMENT_MAGNUS4_GL2, c.data_ptr(), b.PARAMENT_F64, 4, 0.1, U.data_ptr(),
                    b.PARAMENT_PREC_FP64, None)
    assert st == b.PARAMENT_ERR_UNSUPPORTED
    # host memory is refused
    Hh = np.eye(2, dtype=np.complex128)
    st = b.raw_call("parament_propagate_noalloc", 2, 0, Hh.ctypes.data, None, b.PARAMENT_C128, b.PARAMENT_MIDPOINT,
                    None, b.PARAMENT_F64, 4, 0.1, U.data_ptr(), b.PARAMENT_PREC_FP64, None)
    assert st == b.PARAMENT_ERR_INVALID_VALUE
