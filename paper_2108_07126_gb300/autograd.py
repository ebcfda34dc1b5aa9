"""torch.autograd wrapper of the adjoint gradient (parament_propagate_grad).

``gate_infidelity(prop, c, V, dt, prec)`` returns L = 1 - |Tr(V^dagger U(T))|^2 / d^2
for the control samples ``c`` (K, S) on a ``binding.Propagator`` whose Hamiltonians
are set (any integrator; S as in set_controls).  The forward call runs the forward kernels and the adjoint
kernels of the library at once; backward only scales the stored gradient.
"""

from __future__ import annotations

import torch

from .binding import Propagator


class _GateInfidelity(torch.autograd.Function):
    @staticmethod
    def forward(ctx, c: torch.Tensor, prop: Propagator, V: torch.Tensor, dt: float, prec: str):
        prop.set_controls(c.detach(), dt)
        loss, grad = prop.propagate_grad(V, prec)
        ctx.save_for_backward(grad.to(c.dtype))
        return torch.tensor(loss, dtype=c.dtype, device=c.device)

    @staticmethod
    def backward(ctx, g_out):
        (grad,) = ctx.saved_tensors
        return g_out * grad, None, None, None, None


def gate_infidelity(prop: Propagator, c: torch.Tensor, V, dt: float, prec: str = "fp64") -> torch.Tensor:
    return _GateInfidelity.apply(c, prop, torch.as_tensor(V), dt, prec)
