"""Build libparament.so in-tree with nvcc for sm_103a (GB300).

Each translation unit is compiled in parallel to ``_build/*.o`` and linked
into ``libparament.so`` next to this file.  Usage: ``python -m
paper_2108_07126_gb300.build [-v] [--ptxas-info]``.
"""

from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libparament.so")

SOURCES = [
    "pm_api.cu",
    "pm_fused_d2.cu",
    "pm_fused_d4.cu",
    "pm_fused_d8.cu",
    "pm_fused_d16.cu",
    "pm_noalloc.cu",
    "pm_peaks.cu",
    "pm_grad_d2.cu",
    "pm_grad_d4.cu",
    "pm_grad_d8.cu",
    "pm_grad_d16.cu",
    "pm_large_d32.cu",
    "pm_large_d64.cu",
    "pm_large_d128.cu",
    "pm_large_d256.cu",
    "pm_batched_fm.cu",
    "pm_batched_fm_tc.cu",
    "pm_batched_fm_bf.cu",
    "pm_batched_dm.cu",
    "pm_batched_fg.cu",
    "pm_batched_fg_tc.cu",
    "pm_batched_fg_bf.cu",
    "pm_batched_dg.cu",
]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libparament.so")


def _deps() -> list[str]:
    out = [os.path.join(INCLUDE, "parament.h")]
    out += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    return out


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(p) > t for p in [src] + _deps())


def _compile(src: str, ptxas_info: bool) -> tuple[str, str]:
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    path = os.path.join(CSRC, src)
    if not _stale(obj, path) and not ptxas_info:
        return obj, ""
    cmd = [nvcc()] + CFLAGS + (["-Xptxas", "-v"] if ptxas_info else []) + ["-c", path, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return obj, r.stdout + r.stderr


def build(verbose: bool = False, ptxas_info: bool = False, jobs: int | None = None) -> str:
    """Compile and link libparament.so; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    jobs = jobs or min(len(SOURCES), os.cpu_count() or 4)
    with concurrent.futures.ThreadPoolExecutor(jobs) as ex:
        results = list(ex.map(lambda s: _compile(s, ptxas_info), SOURCES))
    objs = [o for o, _ in results]
    if verbose or ptxas_info:
        for (_, log) in results:
            if log:
                print(log, file=sys.stderr)
    if not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        tmp = LIB + ".tmp"
        cmd = [nvcc()] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, ptxas_info="--ptxas-info" in sys.argv))
