"""Tolerances of the GPU parity tests, and a check that can log every measured error.

FP64 path: max-entry |U - U_oracle| <= 1e-11 everywhere.

FP32 and tensor-core paths against the oracle on the float32-rounded inputs (``ref32``): the
slices' products are near-unitary, so every slice adds a rounding error of a few units of
u = 2^-24 to the entries (assembly, polynomial, squarings, leaf product) nearly independently of d,
and the n slice errors add like a random walk: err ~ c u sqrt(n).  Measured on a GB300 over every
FP32 parity case (d = 1..256, n = 1..2^20, all integrators, logged by ``check``), c stays below
6.5 for the CUDA-core products and below 7.7 for 3xTF32 / BF16x3 on the tensor cores.  The bounds
are ``tol32 = 24 u sqrt(n) + 16 u`` (about four times the worst measured c) and twice that for the
tensor-core precisions.  Runs whose slices repeat nearly the same rounding (a drift-dominated
Hamiltonian over many slices) accumulate it coherently instead; they have bounds of their own.

Full-size workloads (exact inputs, so the rounding of the inputs to complex64 counts too) have
bounds of their own, a few times the measured error of each configuration.
"""

import json
import math
import os

TOL64 = 1e-11
U32 = 2.0 ** -24


_last = {}  # arguments of the latest tol32 call, logged beside the next check


def tol32(d, n):
    """FP32 path vs the oracle on float32-rounded inputs, n slices of a d x d problem."""
    _last.update(d=d, n=n)
    return 24.0 * U32 * math.sqrt(max(n, 1)) + 16.0 * U32


def tol_tc(d, n):
    """3xTF32 and split BF16x3 tensor-core products, same comparison."""
    return 2.0 * tol32(d, n)


def check(err, tol, what=""):
    """assert err <= tol; with PARAMENT_ERR_LOG set, also append both to that file (JSON lines)."""
    path = os.environ.get("PARAMENT_ERR_LOG")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"test": os.environ.get("PYTEST_CURRENT_TEST", ""), "what": str(what),
                                "err": float(err), "tol": float(tol), "d": _last.get("d"),
                                "n": _last.get("n")}) + "\n")
    _last.clear()
    assert err <= tol, (what, float(err), float(tol))


# Full-size workloads against the oracle on exact inputs (bounds a few times the measured error;
# the rounding of the inputs to complex64 dominates these errors)
# (measured on a GB300: coupled spins FP32 3.92e-3; dense stress FP32 1.27e-4, 3xTF32 1.04e-3,
# BF16x3 1.34e-3 -- a truncating tensor-core accumulation over the whole k range gave 8.9e-3 and
# must fail; batched sample 9.9e-4 for every form)
FULL_SIZE = {
    "coupled_spins": {"fp32": 8e-3},
    "dense_stress": {"fp32": 4e-4, "fp32_tc_tf32x3": 3e-3, "fp32_tc_bf16x3": 4e-3},
    "batched": {"fp32": 2.5e-3, "fp32_tc_tf32x3": 2.5e-3, "fp32_tc_bf16x3": 2.5e-3},
}

# Coupled spins (drift-dominated, 1.3e5 radians at 2^20 slices) against the FP64 GPU path at 2^18
# slices, default Newton-Schulz step on every leaf product
UNITARY_STEP_2_18 = 2.5e-3
