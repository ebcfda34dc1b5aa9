"""parament_propagate_noalloc through the C ABI, against the context entry point and the oracle.

The no-allocation entry point is for callers that cannot allocate device
memory (an application that owns all device memory through its own
allocator, or a latency-critical loop that cannot afford the synchronisation
of cudaMalloc / cudaFree); it keeps its intermediates in one static device
array.  Each case calls it twice in a row -- the array keeps the previous
call's contents, so the second call checks that the state a call needs is
cleared -- and compares both results with parament_propagate on the same
inputs (1e-11 in FP64; in FP32 the bound of the FP32 parity tests), and one
FP64 case also with the FP64 oracle.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""

import numpy as np
import pytest

import oracle
from paper_2108_07126_gb300 import workloads as wl
from tolerances import TOL64, U32, check, tol32  # noqa: F401

pytestmark = pytest.mark.gpu



CASES = [
    ("coupled_spins", lambda: wl.coupled_spins(n_steps=1 << 14), "fp64"),
    ("coupled_spins", lambda: wl.coupled_spins(n_steps=1 << 14), "fp32"),
    ("random_d5_midpoint", lambda: wl.random_problem(5, 3, 3001, "midpoint", seed=41, g_norm=0.5), "fp64"),
    ("random_d3_simpson", lambda: wl.random_problem(3, 2, 777, "magnus4_simpson", seed=42, g_norm=0.3), "fp32"),
    ("rabi_qubit", lambda: wl.rabi_qubit(), "fp64"),
    # enough slices that the grid reaches PARAMENT_NOALLOC_MAX_BLOCKS (304) blocks, where the
    # partial-product and arrival-counter regions of the array are filled to their size
    ("random_d2_grid_cap", lambda: wl.random_problem(2, 1, 1 << 20, "midpoint", seed=43, g_norm=0.05), "fp64"),
    ("zero_slices", lambda: wl.random_problem(4, 2, 0, "magnus4_gl2", seed=44, g_norm=0.3), "fp64"),
]


def _inputs(prob, prec, hdtype=None):
    import torch

    from paper_2108_07126_gb300 import binding as b

    cdt = hdtype or (torch.complex128 if prec == "fp64" else torch.complex64)
    rdt = torch.float64 if prec == "fp64" else torch.float32
    H0 = torch.as_tensor(prob.H0).to(cdt).cuda().contiguous()
    Hk = torch.as_tensor(prob.Hk).to(cdt).cuda().contiguous()
    c = torch.as_tensor(prob.c).to(rdt).cuda().contiguous()
    dtype = b.PARAMENT_C128 if cdt == torch.complex128 else b.PARAMENT_C64
    cdtype = b.PARAMENT_F64 if prec == "fp64" else b.PARAMENT_F32
    return cdt, H0, Hk, c, dtype, cdtype


def _noalloc(prob, prec, H0, Hk, c, dtype, cdtype, cdt):
    import ctypes

    import torch

    from paper_2108_07126_gb300 import binding as b

    d, K = prob.dim, prob.n_ctrl
    U = torch.full((d, d), float("nan"), dtype=cdt, device="cuda")
    status = ctypes.c_uint32(0xFFFFFFFF)
    st = b.raw_call("parament_propagate_noalloc", d, K, H0.data_ptr(), Hk.data_ptr() if K else None, dtype,
                    b.INTEGRATORS[prob.integrator], c.data_ptr() if c.numel() else None, cdtype, prob.n_steps,
                    prob.dt, U.data_ptr(), b.PRECISIONS[prec], None, ctypes.byref(status))
    assert st == b.PARAMENT_OK, b.parament_status_string(st)
    torch.cuda.synchronize()
    return U.cpu().numpy().astype(np.complex128), status.value


@pytest.mark.parametrize("name,make,prec", CASES, ids=[f"{c[0]}-{c[2]}" for c in CASES])
def test_noalloc_matches_context_entry_point(name, make, prec):
    import torch

    from paper_2108_07126_gb300 import binding as b

    assert torch.cuda.is_available()
    prob = make()
    cdt, H0, Hk, c, dtype, cdtype = _inputs(prob, prec)
    d, K = prob.dim, prob.n_ctrl

    # the existing entry point
    ctx = b.parament_create(0, None)
    try:
        b.parament_set_hamiltonians(ctx, d, K, H0.data_ptr(), Hk.data_ptr() if K else None, dtype,
                                    b.INTEGRATORS[prob.integrator])
        b.parament_set_controls(ctx, c.data_ptr() if c.numel() else None, cdtype, prob.n_steps, prob.dt)
        U_ref = torch.empty(d, d, dtype=cdt, device="cuda")
        b.parament_propagate(ctx, U_ref.data_ptr(), b.PRECISIONS[prec])
        torch.cuda.synchronize()
    finally:
        b.parament_destroy(ctx)
    U_ref = U_ref.cpu().numpy().astype(np.complex128)

    tol = TOL64 if prec == "fp64" else tol32(d, prob.n_steps)
    for call in range(2):
        U, status = _noalloc(prob, prec, H0, Hk, c, dtype, cdtype, cdt)
        assert status == 0, (name, call, status)
        err = np.max(np.abs(U - U_ref))
        check(err, tol, (name, prec, call))
        if prob.n_steps == 0:
            assert np.array_equal(U, np.eye(d)), (name, call)


def test_noalloc_fp64_matches_oracle():
    """FP64 against the oracle's eigendecomposition product (Sec. 2, Eq. slices), all three integrators."""
    for integ, seed in (("midpoint", 51), ("magnus4_gl2", 52), ("magnus4_simpson", 53)):
        prob = wl.random_problem(7, 3, 1500, integ, seed=seed, g_norm=0.4)
        ref = oracle.propagate(prob.H0, prob.Hk, prob.c, prob.dt, prob.integrator)
        cdt, H0, Hk, c, dtype, cdtype = _inputs(prob, "fp64")
        for call in range(2):
            U, status = _noalloc(prob, "fp64", H0, Hk, c, dtype, cdtype, cdt)
            assert status == 0
            err = float(np.max(np.abs(U - ref)))
            assert err <= TOL64, (integ, call, err)


def test_noalloc_complex64_storage_with_fp64_arithmetic():
    """complex64 Hamiltonians and U with FP64 arithmetic and FP64 controls: the oracle on the rounded inputs."""
    import torch

    prob = wl.random_problem(6, 2, 999, "magnus4_gl2", seed=54, g_norm=0.3)
    cdt, H0, Hk, c, dtype, cdtype = _inputs(prob, "fp64", hdtype=torch.complex64)
    ref = oracle.propagate(prob.H0.astype(np.complex64).astype(np.complex128),
                           prob.Hk.astype(np.complex64).astype(np.complex128), prob.c, prob.dt, prob.integrator)
    for call in range(2):
        U, status = _noalloc(prob, "fp64", H0, Hk, c, dtype, cdtype, cdt)
        assert status == 0
        # only the final rounding of U to complex64 separates the two
        err = float(np.max(np.abs(U - ref)))
        assert err <= 4 * U32, (call, err)


def test_noalloc_reports_nonfinite_controls():
    """A NaN control sample reaches the FP64 norm bound: the device status word says so."""
    from paper_2108_07126_gb300 import binding as b

    prob = wl.random_problem(4, 2, 300, "midpoint", seed=55, g_norm=0.3)
    cdt, H0, Hk, c, dtype, cdtype = _inputs(prob, "fp64")
    c[1, 17] = float("nan")
    _, status = _noalloc(prob, "fp64", H0, Hk, c, dtype, cdtype, cdt)
    assert status & b.PARAMENT_DEV_NONFINITE_NORM
    # the next call with clean inputs starts from a cleared status word
    c[1, 17] = 0.0
    _, status = _noalloc(prob, "fp64", H0, Hk, c, dtype, cdtype, cdt)
    assert status == 0


def test_noalloc_rejects_what_it_cannot_hold():
    import torch

    from paper_2108_07126_gb300 import binding as b

    def call(d, K, H, Hk, dtype, integ, c, cdtype, n, dt, U, prec):
        return b.raw_call("parament_propagate_noalloc", d, K, H, Hk, dtype, integ, c, cdtype, n, dt, U, prec,
                          None, None)

    # d beyond the array's limit: UNSUPPORTED; d < 1: INVALID_VALUE
    H = torch.eye(32, dtype=torch.complex128, device="cuda")
    U = torch.empty(32, 32, dtype=torch.complex128, device="cuda")
    st = call(32, 0, H.data_ptr(), None, b.PARAMENT_C128, b.PARAMENT_MIDPOINT, None, b.PARAMENT_F64, 4, 0.1,
              U.data_ptr(), b.PARAMENT_PREC_FP64)
    assert st == b.PARAMENT_ERR_UNSUPPORTED
    st = call(0, 0, H.data_ptr(), None, b.PARAMENT_C128, b.PARAMENT_MIDPOINT, None, b.PARAMENT_F64, 4, 0.1,
              U.data_ptr(), b.PARAMENT_PREC_FP64)
    assert st == b.PARAMENT_ERR_INVALID_VALUE
    # nine controls with a Magnus integrator need 1 + 9 * 12 / 2 = 55 > 45 basis matrices
    H = torch.eye(2, dtype=torch.complex128, device="cuda")
    Hk = torch.zeros(9, 2, 2, dtype=torch.complex128, device="cuda")
    c = torch.zeros(9, 8, dtype=torch.float64, device="cuda")
    U = torch.empty(2, 2, dtype=torch.complex128, device="cuda")
    st = call(2, 9, H.data_ptr(), Hk.data_ptr(), b.PARAMENT_C128, b.PARAMENT_MAGNUS4_GL2, c.data_ptr(),
              b.PARAMENT_F64, 4, 0.1, U.data_ptr(), b.PARAMENT_PREC_FP64)
    assert st == b.PARAMENT_ERR_UNSUPPORTED
    # tensor-core precisions are not available here
    st = call(2, 0, H.data_ptr(), None, b.PARAMENT_C64, b.PARAMENT_MIDPOINT, None, b.PARAMENT_F32, 4, 0.1,
              U.data_ptr(), b.PARAMENT_PREC_FP32_TC_TF32X3)
    assert st == b.PARAMENT_ERR_UNSUPPORTED
    # host memory is refused
    Hh = np.eye(2, dtype=np.complex128)
    st = call(2, 0, Hh.ctypes.data, None, b.PARAMENT_C128, b.PARAMENT_MIDPOINT, None, b.PARAMENT_F64, 4, 0.1,
              U.data_ptr(), b.PARAMENT_PREC_FP64)
    assert st == b.PARAMENT_ERR_INVALID_VALUE
    # an unknown control dtype, and a control dtype that does not match the precision
    Hk1 = torch.zeros(1, 2, 2, dtype=torch.complex128, device="cuda")
    c1 = torch.zeros(1, 4, dtype=torch.float64, device="cuda")
    for cdtype, prec in ((7, b.PARAMENT_PREC_FP32), (b.PARAMENT_F32, b.PARAMENT_PREC_FP64)):
        st = call(2, 1, H.data_ptr(), Hk1.data_ptr(), b.PARAMENT_C128, b.PARAMENT_MIDPOINT, c1.data_ptr(), cdtype, 4,
                  0.1, U.data_ptr(), prec)
        assert st == b.PARAMENT_ERR_INVALID_VALUE, (cdtype, prec)
    # a non-finite slice duration
    st = call(2, 1, H.data_ptr(), Hk1.data_ptr(), b.PARAMENT_C128, b.PARAMENT_MIDPOINT, c1.data_ptr(),
              b.PARAMENT_F64, 4, float("inf"), U.data_ptr(), b.PARAMENT_PREC_FP64)
    assert st == b.PARAMENT_ERR_NONFINITE
    # misaligned U (complex128 needs 16 bytes) and misaligned FP64 controls (8 bytes); nothing is launched
    Ubig = torch.zeros(5, dtype=torch.complex128, device="cuda")
    st = call(2, 1, H.data_ptr(), Hk1.data_ptr(), b.PARAMENT_C128, b.PARAMENT_MIDPOINT, c1.data_ptr(),
              b.PARAMENT_F64, 4, 0.1, Ubig.data_ptr() + 8, b.PARAMENT_PREC_FP64)
    assert st == b.PARAMENT_ERR_INVALID_VALUE
    cbig = torch.zeros(1, 8, dtype=torch.float64, device="cuda")
    st = call(2, 1, H.data_ptr(), Hk1.data_ptr(), b.PARAMENT_C128, b.PARAMENT_MIDPOINT, cbig.data_ptr() + 4,
              b.PARAMENT_F64, 4, 0.1, U.data_ptr(), b.PARAMENT_PREC_FP64)
    assert st == b.PARAMENT_ERR_INVALID_VALUE
    torch.cuda.synchronize()
