"""FP64 CPU oracle (test infrastructure only; see ``parament_oracle``)."""

from .parament_oracle import *  # noqa: F401,F403
from .parament_oracle import (  # noqa: F401
    INTEGRATORS,
    MAGNUS4_GL2,
    MAGNUS4_SIMPSON,
    MIDPOINT,
    commutator,
    effective_control_count,
    exact_slice_propagators,
    exponent_derivatives,
    frechet_exp,
    frechet_phi,
    gate_loss,
    hamiltonian,
    loss_and_gradient,
    ordered_product,
    propagate,
    samples_per_run,
    slice_exponents,
    trajectory,
    trajectory_times,
)
