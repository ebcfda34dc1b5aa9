"""The FP64 oracle's U(T) computed on several host cores.

TEST INFRASTRUCTURE ONLY (imported by the tests and by the benchmark's CPU-baseline and error
legs; never by the library).  The slices are cut into contiguous ranges; each range is propagated
by ``parament_oracle.propagate`` (unchanged) in its own process, and the partial products are
multiplied in time order, later ranges on the left (Sec. 2, Eq. slices: U(T) = U_N ... U_1 =
P_last ... P_first).  Only the association of the product differs from the single-process oracle,
which changes the FP64 result at the level of rounding.
"""

from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

from .parament_oracle import MAGNUS4_GL2, MAGNUS4_SIMPSON, MIDPOINT, propagate


def sample_range(a: int, b: int, integrator: str) -> slice:
    """Control samples that slices [a, b) read: midpoint one per slice, Gauss-Legendre two per
    slice, Simpson the end points and centres, end points shared with the neighbours."""
    if integrator == MIDPOINT:
        return slice(a, b)
    if integrator == MAGNUS4_GL2:
        return slice(2 * a, 2 * b)
    if integrator == MAGNUS4_SIMPSON:
        return slice(2 * a, 2 * b + 1)
    raise ValueError(f"unknown integrator {integrator!r}")


def _range_product(args):
    H0, Hk, c, dt, integrator = args
    return propagate(H0, Hk, c, dt, integrator)


def propagate_parallel(H0, Hk, c, dt: float, integrator: str = MIDPOINT, workers: int = 0) -> np.ndarray:
    """U(T) of ``propagate`` with the slices split over ``workers`` processes (0 = every host core).

    Worker processes are started with ``spawn`` (safe after a CUDA context exists in the caller)
    and run single-threaded BLAS.
    """
    c = np.asarray(c, dtype=np.float64)
    S = c.shape[1] if c.ndim == 2 and c.shape[0] > 0 else None
    if integrator == MIDPOINT:
        n = S
    elif integrator == MAGNUS4_GL2:
        n = None if S is None else S // 2
    else:
        n = None if S is None else (S - 1) // 2
    if n is None:
        raise ValueError("propagate_parallel needs at least one control to count the slices")
    workers = max(1, min(workers or (os.cpu_count() or 1), n))
    if workers == 1 or n < 64:
        return propagate(H0, Hk, c, dt, integrator)
    cuts = [n * w // workers for w in range(workers + 1)]
    jobs = [(H0, Hk, np.ascontiguousarray(c[:, sample_range(cuts[w], cuts[w + 1], integrator)]), dt, integrator)
            for w in range(workers)]
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(workers) as pool:
            parts = pool.map(_range_product, jobs)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    U = parts[0]
    for P in parts[1:]:
        U = P @ U  # later slices on the left
    return U
