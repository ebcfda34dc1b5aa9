"""Thin ctypes binding of libparament.so (include/parament.h).

The functions keep the C names and take the same arguments (device or host
pointers as Python ints); they only marshal arguments and turn a non-zero
status into ``ParamentError``.  Every step of the propagation runs in the CUDA
library.  Importing this module fails loudly if the library has not been
built -- there is no CPU fallback.

``Propagator`` wraps one context for torch tensors: it passes ``data_ptr()``
values and the current torch CUDA stream.
"""

from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libparament.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it with `python -m paper_2108_07126_gb300.build` "
        "(the propagator has no CPU fallback)")

_lib = ctypes.CDLL(LIB_PATH)

# ---- enums (parament.h)
PARAMENT_OK = 0
PARAMENT_ERR_INVALID_VALUE = 1
PARAMENT_ERR_STATE = 2
PARAMENT_ERR_ALLOC = 3
PARAMENT_ERR_CUDA = 4
PARAMENT_ERR_NONFINITE = 5
PARAMENT_ERR_NOT_HERMITIAN = 6
PARAMENT_ERR_TIMEOUT = 7
PARAMENT_ERR_UNSUPPORTED = 8

PARAMENT_C64 = 0
PARAMENT_C128 = 1
PARAMENT_F32 = 0
PARAMENT_F64 = 1

PARAMENT_MIDPOINT = 0
PARAMENT_MAGNUS4_GL2 = 1
PARAMENT_MAGNUS4_SIMPSON = 2

PARAMENT_PREC_FP64 = 0
PARAMENT_PREC_FP32 = 1
PARAMENT_PREC_FP32_TC_BF16X3 = 2
PARAMENT_PREC_FP32_TC_TF32X3 = 3

PARAMENT_OPT_TAYLOR_DEGREE = 1
PARAMENT_OPT_GRID_BLOCKS = 2
PARAMENT_OPT_BLOCK_WARPS = 3
PARAMENT_OPT_CHECK_HERMITIAN = 4
PARAMENT_OPT_EXTRA_SQUARINGS = 5
PARAMENT_OPT_HERMITIAN_TOL_E12 = 7
PARAMENT_OPT_GRAD_SUBCHUNK = 8
PARAMENT_OPT_WORKSPACE_MB = 9
PARAMENT_OPT_BATCH_LEAF_STEPS = 10
PARAMENT_OPT_BATCH_ITEMS_PER_SM = 11
PARAMENT_OPT_BATCH_GRAPH = 12
PARAMENT_OPT_EXP_METHOD = 13
PARAMENT_OPT_UNITARY_STEP = 14
PARAMENT_OPT_BATCH_CUDA_CORE_CLASSES = 15

PARAMENT_DEV_NONFINITE_NORM = 0x1
PARAMENT_DEV_NORM_CAPPED = 0x2
PARAMENT_DEV_TENSOR_TIMEOUT = 0x4

PARAMENT_BACKEND_CUDA_CORES = 0x1
PARAMENT_BACKEND_MMA_SYNC = 0x2
PARAMENT_BACKEND_TCGEN05 = 0x4

INTEGRATORS = {"midpoint": PARAMENT_MIDPOINT, "magnus4_gl2": PARAMENT_MAGNUS4_GL2,
               "magnus4_simpson": PARAMENT_MAGNUS4_SIMPSON}
PRECISIONS = {"fp64": PARAMENT_PREC_FP64, "fp32": PARAMENT_PREC_FP32,
              "fp32_tc_bf16x3": PARAMENT_PREC_FP32_TC_BF16X3, "fp32_tc_tf32x3": PARAMENT_PREC_FP32_TC_TF32X3}


class parament_stats(ctypes.Structure):
    _fields_ = [
        ("n_steps", ctypes.c_int64),
        ("dim", ctypes.c_int32),
        ("n_basis", ctypes.c_int32),
        ("grid_blocks", ctypes.c_int32),
        ("block_threads", ctypes.c_int32),
        ("leaves", ctypes.c_int32),
        ("max_degree", ctypes.c_int32),
        ("max_squarings", ctypes.c_int32),
        ("grad_subchunk", ctypes.c_int32),
        ("exp_products", ctypes.c_int64),
        ("tree_products", ctypes.c_int64),
        ("device_status", ctypes.c_uint32),
        ("product_backends", ctypes.c_uint32),
        ("kernel_ms", ctypes.c_double),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_ if not name.startswith("reserved")}


class parament_peaks(ctypes.Structure):
    _fields_ = [
        ("fp32_tflops", ctypes.c_double),
        ("fp64_tflops", ctypes.c_double),
        ("tf32_tflops", ctypes.c_double),
        ("bf16_tflops", ctypes.c_double),
        ("sm_count", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("max_sm_clock_mhz", ctypes.c_double),
        ("fp32_tflops_max_clock", ctypes.c_double),
        ("fp64_tflops_max_clock", ctypes.c_double),
    ]


class parament_instance(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("n_ctrl", ctypes.c_int),
        ("H0", ctypes.c_void_p),
        ("Hk", ctypes.c_void_p),
        ("c", ctypes.c_void_p),
        ("n_steps", ctypes.c_int64),
        ("dt", ctypes.c_double),
        ("U_out", ctypes.c_void_p),
    ]


_vp = ctypes.c_void_p
_SIGS = {
    "parament_version": ([], ctypes.c_int),
    "parament_create": ([ctypes.POINTER(_vp), ctypes.c_int, _vp], ctypes.c_int),
    "parament_destroy": ([_vp], ctypes.c_int),
    "parament_set_stream": ([_vp, _vp], ctypes.c_int),
    "parament_set_hamiltonians": ([_vp, ctypes.c_int, ctypes.c_int, _vp, _vp, ctypes.c_int, ctypes.c_int],
                                  ctypes.c_int),
    "parament_set_controls": ([_vp, _vp, ctypes.c_int, ctypes.c_int64, ctypes.c_double], ctypes.c_int),
    "parament_propagate": ([_vp, _vp, ctypes.c_int], ctypes.c_int),
    "parament_propagate_grad": ([_vp, _vp, ctypes.POINTER(ctypes.c_double), _vp, _vp, ctypes.c_int], ctypes.c_int),
    "parament_propagate_trajectory": ([_vp, _vp, _vp, ctypes.c_int64, ctypes.c_int], ctypes.c_int),
    "parament_get_stats": ([_vp, ctypes.POINTER(parament_stats)], ctypes.c_int),
    "parament_set_option": ([_vp, ctypes.c_int, ctypes.c_int64], ctypes.c_int),
    "parament_get_option": ([_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "parament_taylor_theta": ([ctypes.c_int, ctypes.c_double], ctypes.c_double),
    "parament_taylor_choice": ([ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "parament_propagate_noalloc": ([ctypes.c_int, ctypes.c_int, _vp, _vp, ctypes.c_int, ctypes.c_int, _vp,
                                    ctypes.c_int, ctypes.c_int64, ctypes.c_double, _vp, ctypes.c_int, _vp,
                                    ctypes.POINTER(ctypes.c_uint32)], ctypes.c_int),
    "parament_propagate_batched": ([_vp, ctypes.POINTER(parament_instance), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "parament_batch_autotune": ([_vp, ctypes.POINTER(parament_instance), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                 ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(ctypes.c_uint32)], ctypes.c_int),
    "parament_measure_peaks": ([ctypes.c_int, _vp, ctypes.POINTER(parament_peaks)], ctypes.c_int),
    "parament_chebyshev_theta": ([ctypes.c_int, ctypes.c_double], ctypes.c_double),
    "parament_chebyshev_degree": ([ctypes.c_double, ctypes.c_double], ctypes.c_int),
    "parament_bessel_j": ([ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "parament_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "parament_last_error": ([_vp], ctypes.c_char_p),
}
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res


class ParamentError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{parament_status_string(status)}: {message}")
        self.status = status


def _check(status: int, ctx=None) -> None:
    if status != PARAMENT_OK:
        raise ParamentError(status, parament_last_error(ctx) if ctx else "")


# ---- C-named wrappers -------------------------------------------------------------------

def parament_version() -> int:
    return _lib.parament_version()


def parament_status_string(status: int) -> str:
    return _lib.parament_status_string(int(status)).decode()


def parament_last_error(ctx) -> str:
    return _lib.parament_last_error(ctx).decode()


def parament_create(device: int = 0, stream: int | None = None):
    h = _vp()
    _check(_lib.parament_create(ctypes.byref(h), int(device), stream or None))
    return h


def parament_destroy(ctx) -> None:
    _check(_lib.parament_destroy(ctx))


def parament_set_stream(ctx, stream: int | None) -> None:
    _check(_lib.parament_set_stream(ctx, stream or None), ctx)


def parament_set_hamiltonians(ctx, dim: int, n_ctrl: int, H0_ptr: int, Hk_ptr: int | None, dtype: int,
                              integrator: int) -> None:
    _check(_lib.parament_set_hamiltonians(ctx, int(dim), int(n_ctrl), H0_ptr, Hk_ptr or None, int(dtype),
                                          int(integrator)), ctx)


def parament_set_controls(ctx, c_ptr: int | None, cdtype: int, n_steps: int, dt: float) -> None:
    _check(_lib.parament_set_controls(ctx, c_ptr or None, int(cdtype), int(n_steps), float(dt)), ctx)


def parament_propagate(ctx, U_ptr: int, prec: int) -> None:
    _check(_lib.parament_propagate(ctx, U_ptr, int(prec)), ctx)


def parament_propagate_grad(ctx, V_ptr: int, grad_ptr: int, U_ptr: int | None, prec: int,
                            want_loss: bool = True) -> float | None:
    loss = ctypes.c_double(float("nan"))
    _check(_lib.parament_propagate_grad(ctx, V_ptr, ctypes.byref(loss) if want_loss else None, grad_ptr,
                                        U_ptr or None, int(prec)), ctx)
    return loss.value if want_loss else None


def parament_propagate_trajectory(ctx, psi0_ptr: int | None, out_ptr: int | None, every: int, prec: int) -> None:
    _check(_lib.parament_propagate_trajectory(ctx, psi0_ptr or None, out_ptr or None, int(every), int(prec)), ctx)


def parament_get_stats(ctx) -> dict:
    s = parament_stats()
    _check(_lib.parament_get_stats(ctx, ctypes.byref(s)), ctx)
    return s.as_dict()


def parament_set_option(ctx, key: int, value: int) -> None:
    _check(_lib.parament_set_option(ctx, int(key), int(value)), ctx)


def parament_get_option(ctx, key: int) -> int:
    v = ctypes.c_int64()
    _check(_lib.parament_get_option(ctx, int(key), ctypes.byref(v)), ctx)
    return v.value


def parament_taylor_theta(m: int, u: float) -> float:
    return _lib.parament_taylor_theta(int(m), float(u))


def parament_taylor_choice(norm_bound: float, u: float, force_m: int = 0) -> tuple[int, int]:
    m = ctypes.c_int()
    s = ctypes.c_int()
    _check(_lib.parament_taylor_choice(float(norm_bound), float(u), int(force_m), ctypes.byref(m), ctypes.byref(s)))
    return m.value, s.value


def parament_propagate_noalloc(dim: int, n_ctrl: int, H0_ptr: int, Hk_ptr: int | None, dtype: int, integrator: int,
                               c_ptr: int | None, cdtype: int, n_steps: int, dt: float, U_ptr: int, prec: int,
                               stream: int | None = None, wait_status: bool = False) -> int | None:
    """One propagation that allocates nothing (device pointers only; see parament.h).

    With ``wait_status`` the call waits and returns the PARAMENT_DEV_* bits of the kernel.
    """
    st = ctypes.c_uint32(0)
    _check(_lib.parament_propagate_noalloc(int(dim), int(n_ctrl), H0_ptr, Hk_ptr or None, int(dtype),
                                           int(integrator), c_ptr or None, int(cdtype), int(n_steps), float(dt),
                                           U_ptr, int(prec), stream or None,
                                           ctypes.byref(st) if wait_status else None))
    return st.value if wait_status else None


def _instances(inst):
    arr = (parament_instance * max(len(inst), 1))()
    for i, q in enumerate(inst):
        arr[i] = q
    return arr


def parament_propagate_batched(ctx, inst: list, dtype: int, cdtype: int, integrator: int, prec: int) -> None:
    arr = _instances(inst)
    _check(_lib.parament_propagate_batched(ctx, arr, len(inst), int(dtype), int(cdtype), int(integrator),
                                           int(prec)), ctx)


def parament_batch_autotune(ctx, inst: list, dtype: int, cdtype: int, integrator: int, prec: int):
    arr = _instances(inst)
    l, i, ms, m = ctypes.c_int(), ctypes.c_int(), ctypes.c_double(), ctypes.c_uint32()
    _check(_lib.parament_batch_autotune(ctx, arr, len(inst), int(dtype), int(cdtype), int(integrator), int(prec),
                                        ctypes.byref(l), ctypes.byref(i), ctypes.byref(ms), ctypes.byref(m)), ctx)
    return l.value, i.value, ms.value, m.value


def parament_measure_peaks(device: int = 0, stream: int | None = None) -> dict:
    """Measured FP32 / FP64 FMA and TF32 / BF16 tcgen05 rates of the device (TFLOP/s)."""
    pk = parament_peaks()
    _check(_lib.parament_measure_peaks(int(device), stream or None, ctypes.byref(pk)))
    return {name: getattr(pk, name) for name, _ in pk._fields_ if name != "reserved"}


def parament_chebyshev_theta(m: int, u: float) -> float:
    return _lib.parament_chebyshev_theta(int(m), float(u))


def parament_chebyshev_degree(half_width: float, u: float) -> int:
    return _lib.parament_chebyshev_degree(float(half_width), float(u))


def parament_bessel_j(n: int, x: float) -> list:
    out = (ctypes.c_double * (n + 1))()
    _check(_lib.parament_bessel_j(int(n), float(x), out))
    return list(out)


def raw_call(name: str, *args) -> int:
    """Call a C entry point directly and return its status (for tests of the error paths)."""
    return getattr(_lib, name)(*args)


# ---- torch convenience wrapper ------------------------------------------------------------

class Propagator:
    """One library context bound to a CUDA device and the current torch stream.

    ``set_hamiltonians(H0, Hk, integrator)`` takes complex64/complex128 tensors or
    arrays; ``set_controls(c, dt)`` a real (K, S) tensor; ``propagate(prec)``
    returns U(T) as a device tensor of the Hamiltonians' dtype.
    """

    def __init__(self, device: int = 0):
        import torch

        self._torch = torch
        self.device = torch.device("cuda", device)
        self.ctx = parament_create(device, torch.cuda.current_stream(self.device).cuda_stream)
        self._keep = []
        self.dim = None
        self.cdtype = None

    def close(self):
        if self.ctx is not None:
            parament_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _sync_stream(self):
        parament_set_stream(self.ctx, self._torch.cuda.current_stream(self.device).cuda_stream)

    def set_option(self, key: int, value: int):
        parament_set_option(self.ctx, key, value)

    def get_option(self, key: int) -> int:
        return parament_get_option(self.ctx, key)

    def set_hamiltonians(self, H0, Hk, integrator: str = "midpoint"):
        torch = self._torch
        H0 = torch.as_tensor(H0)
        if H0.dtype not in (torch.complex64, torch.complex128):
            H0 = H0.to(torch.complex128)
        d = H0.shape[-1]
        Hk = torch.as_tensor(Hk).to(H0.dtype).reshape(-1, d, d) if Hk is not None else torch.zeros(0, d, d,
                                                                                               dtype=H0.dtype)
        H0 = H0.to(self.device).contiguous()
        Hk = Hk.to(self.device).contiguous()
        self._sync_stream()
        parament_set_hamiltonians(self.ctx, d, Hk.shape[0], H0.data_ptr(), Hk.data_ptr() if Hk.numel() else None,
                                  PARAMENT_C128 if H0.dtype == torch.complex128 else PARAMENT_C64,
                                  INTEGRATORS[integrator])
        self.dim = d
        self.dtype = H0.dtype
        self.n_ctrl = Hk.shape[0]
        self.integrator = integrator
        self._keep = [H0, Hk]

    def set_controls(self, c, dt: float, n_steps: int | None = None):
        torch = self._torch
        c = torch.as_tensor(c)
        if c.dtype not in (torch.float32, torch.float64):
            c = c.to(torch.float64)
        c = c.to(self.device).contiguous()
        if n_steps is None:
            S = c.shape[-1] if c.numel() else 0
            n_steps = {"midpoint": S, "magnus4_gl2": S // 2, "magnus4_simpson": max(S - 1, 0) // 2}[self.integrator]
        self._sync_stream()
        parament_set_controls(self.ctx, c.data_ptr() if c.numel() else None,
                              PARAMENT_F64 if c.dtype == torch.float64 else PARAMENT_F32, n_steps, dt)
        self._ctrl = c
        self.n_steps = n_steps

    def propagate(self, prec: str = "fp64", out=None):
        torch = self._torch
        if out is None:
            out = torch.empty(self.dim, self.dim, dtype=self.dtype, device=self.device)
        self._sync_stream()
        parament_propagate(self.ctx, out.data_ptr(), PRECISIONS[prec])
        return out

    def propagate_trajectory(self, prec: str = "fp64", every: int = 1, psi0=None, out=None):
        """U(t_n) (n_out, d, d), or psi(t_n) = U(t_n) psi0 (n_out, d), after slices every, 2 every, ..., N."""
        torch = self._torch
        n_out = -(-self.n_steps // every) if every > 0 else 0
        psi = None
        if psi0 is not None:
            psi = torch.as_tensor(psi0).to(self.dtype).to(self.device).contiguous()
        if out is None:
            shape = (n_out, self.dim) if psi is not None else (n_out, self.dim, self.dim)
            out = torch.empty(shape, dtype=self.dtype, device=self.device)
        self._sync_stream()
        parament_propagate_trajectory(self.ctx, psi.data_ptr() if psi is not None else None,
                                      out.data_ptr() if out.numel() else None, every, PRECISIONS[prec])
        return out

    def propagate_grad(self, V, prec: str = "fp64", want_U: bool = False):
        """Loss 1 - |Tr(V^dagger U)|^2 / d^2, its gradient (K, S) w.r.t. the control samples, optionally U."""
        torch = self._torch
        V = torch.as_tensor(V).to(self.dtype).to(self.device).contiguous()
        rdt = torch.float64 if prec == "fp64" else torch.float32
        S = {"midpoint": self.n_steps, "magnus4_gl2": 2 * self.n_steps,
             "magnus4_simpson": 2 * self.n_steps + 1}[self.integrator]
        grad = torch.empty(self.n_ctrl, S, dtype=rdt, device=self.device)
        U = torch.empty(self.dim, self.dim, dtype=self.dtype, device=self.device) if want_U else None
        self._sync_stream()
        loss = parament_propagate_grad(self.ctx, V.data_ptr(), grad.data_ptr(), U.data_ptr() if want_U else None,
                                       PRECISIONS[prec])
        return (loss, grad, U) if want_U else (loss, grad)

    def batch(self, problems, prec: str = "fp32", integrator: str = "midpoint"):
        """Device-resident tensors and instance records for a batched call.

        ``problems``: iterable of (H0, Hk, c, dt, n_steps).  Returns (instances, keep, outputs); ``keep``
        holds the tensors the records point to.
        """
        torch = self._torch
        cdt = torch.complex128 if prec == "fp64" else torch.complex64
        rdt = torch.float64 if prec == "fp64" else torch.float32
        inst, keep, outs = [], [], []
        for (H0, Hk, c, dt, n) in problems:
            H0t = torch.as_tensor(H0).to(cdt).to(self.device).contiguous()
            d = H0t.shape[-1]
            Hkt = torch.as_tensor(Hk).to(cdt).to(self.device).reshape(-1, d, d).contiguous()
            ct = torch.as_tensor(c).to(rdt).to(self.device).contiguous()
            U = torch.empty(d, d, dtype=cdt, device=self.device)
            keep += [H0t, Hkt, ct]
            outs.append(U)
            inst.append(parament_instance(d, Hkt.shape[0], H0t.data_ptr(), Hkt.data_ptr() if Hkt.numel() else None,
                                          ct.data_ptr() if ct.numel() else None, int(n), float(dt), U.data_ptr()))
        return inst, keep, outs

    def propagate_batched(self, inst, prec: str = "fp32", integrator: str = "midpoint"):
        torch = self._torch
        self._sync_stream()
        parament_propagate_batched(self.ctx, inst, PARAMENT_C128 if prec == "fp64" else PARAMENT_C64,
                                   PARAMENT_F64 if prec == "fp64" else PARAMENT_F32, INTEGRATORS[integrator],
                                   PRECISIONS[prec])

    def batch_autotune(self, inst, prec: str = "fp32", integrator: str = "midpoint"):
        self._sync_stream()
        return parament_batch_autotune(self.ctx, inst, PARAMENT_C128 if prec == "fp64" else PARAMENT_C64,
                                       PARAMENT_F64 if prec == "fp64" else PARAMENT_F32, INTEGRATORS[integrator],
                                       PRECISIONS[prec])

    def stats(self) -> dict:
        return parament_get_stats(self.ctx)
