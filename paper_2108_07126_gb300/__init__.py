"""GB300-native parallel-in-time propagator (arXiv 2108.07126, PARAMENT).

The CUDA library ``libparament.so`` (C ABI in ``include/parament.h``) does
all of the work; ``binding`` is its ctypes binding and is imported lazily so
that ``workloads`` (numpy input generators) is usable without a build.
"""

import importlib

__all__ = ["binding", "workloads", "build"]


def __getattr__(name):
    if name in ("binding", "workloads", "build"):
        return importlib.import_module(f"{__name__}.{name}")
    b = importlib.import_module(f"{__name__}.binding")
    if hasattr(b, name):
        return getattr(b, name)
    raise AttributeError(name)
