"""Build the CUDA library in-tree: ``paper_2605_26388_b300/_lib/libdgsem.so`` (sm_103a).

Run ``python -m paper_2605_26388_b300.build`` or call :func:`build_library`.  The compiled
``.so`` stays inside the package directory so that it travels with the source tree.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libdgsem.so")
SOURCES = ["dg_api.cu", "dg_kernels.cu", "dg_stage2d.cu", "dg_stage3d.cu", "dg_batched2d.cu",
           "dg_batched3d.cu", "dg_adjoint.cu", "dg_adjoint_ec.cu", "dg_noalloc.cu", "dg_reacting.cu",
           "dg_shock.cu", "dg_curved.cu", "dg_peaks.cu"]
HEADERS = ["dg_device.cuh", "dg_internal.h", "dg_stage.cuh", "dg_batched.cuh", "dg_stage_ec3.cuh",
           "dg_adjoint.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    deps.append(os.path.join(os.path.dirname(HERE), "include", "dgsem.h"))
    return any(os.path.getmtime(d) > t for d in deps)


def build_library(force: bool = False, verbose: bool = False) -> str:
    """Compile every translation unit with nvcc (CUDA 13, -O3 -lineinfo, sm_103a) in
    parallel, then link them into one shared library."""
    if not force and not _stale():
        return LIB
    os.makedirs(LIBDIR, exist_ok=True)
    nvcc = os.environ.get("NVCC", "nvcc")
    objdir = os.path.join(LIBDIR, "obj")
    os.makedirs(objdir, exist_ok=True)
    flags = [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler",
             "-fvisibility=hidden", "--expt-relaxed-constexpr"]
    if verbose:
        flags.append("-Xptxas=-v")
    procs, objs = [], []
    hdr_t = max(os.path.getmtime(d) for d in [os.path.join(CSRC, h) for h in HEADERS] +
                [os.path.join(os.path.dirname(HERE), "include", "dgsem.h")])
    for f in SOURCES:
        obj = os.path.join(objdir, f.replace(".cu", ".o"))
        objs.append(obj)
        src = os.path.join(CSRC, f)
        # recompile an object older than its source or than any shared header
        if not force and os.path.exists(obj) and os.path.getmtime(obj) > max(os.path.getmtime(src), hdr_t):
            continue
        procs.append((f, subprocess.Popen([nvcc, *flags, "-c", src, "-o", obj])))
    failed = [f for f, p in procs if p.wait() != 0]
    if failed:
        raise subprocess.CalledProcessError(1, f"nvcc {failed}")
    subprocess.run([nvcc, *ARCH, "-shared", "-o", LIB + ".tmp", *objs], check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build_library(force="--force" in sys.argv, verbose="-v" in sys.argv))
