"""Build the CUDA library (libartsim.so) in-tree with nvcc for sm_103a.

Five translation units compiled in parallel with ``-gencode arch=compute_103a,code=sm_103a``
(the per-type kernels with shared-memory rows, with global-memory rows, the persistent kernel, the
step-derivative kernel, and the C ABI), then linked into one shared library; the CUDA runtime is linked statically so the
library has no dependency beyond the driver.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB_PATH = os.path.join(HERE, "libartsim.so")
UNITS = ("kernels_shared.cu", "kernels_global.cu", "kernels_persistent.cu", "kernels_adjoint.cu", "kernels_tape.cu",
         "sim_api.cu")
SOURCES = [os.path.join(CSRC, f) for f in UNITS + ("step_kernel.cuh", "tangent_step.cuh", "adjoint_kernel.cuh", "sim_internal.h",
                                                   "launch.h")] + \
    [os.path.join(INCLUDE, "sim.h"), os.path.abspath(__file__)]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMPILE_FLAGS = ARCH + ["-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC"]
# The step kernels divide and take square roots with the approximate forms (a few ulp) instead
# of the IEEE-rounded sequences, which sit on the Cholesky pivot chain and in the articulated-body
# sweeps (humanoid and hand steps 4-5 % faster); the FP32 results move by far less than the
# tolerance the parity tests derive from the FP32 conditioning of each step. The derivative
# kernel and the host code keep IEEE division and square root.
STEP_UNITS = ("kernels_shared.cu", "kernels_global.cu", "kernels_persistent.cu")
STEP_FLAGS = ["-prec-div=false", "-prec-sqrt=false"]
LINK_FLAGS = ARCH + ["-shared", "-cudart", "static"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libartsim.so")


def build_library(force: bool = False, verbose: bool = False) -> str:
    stale = not os.path.exists(LIB_PATH) or any(os.path.getmtime(s) > os.path.getmtime(LIB_PATH) for s in SOURCES)
    if not (force or stale):
        return LIB_PATH
    tag = f".tmp{os.getpid()}"
    objs = [os.path.join(CSRC, u[:-3] + tag + ".o") for u in UNITS]

    def compile_unit(i):
        cmd = [nvcc()] + COMPILE_FLAGS + (STEP_FLAGS if UNITS[i] in STEP_UNITS else []) + \
            (["-Xptxas", "-v"] if verbose else []) + ["-c", "-o", objs[i], os.path.join(CSRC, UNITS[i])]
        return subprocess.run(cmd, capture_output=True, text=True)

    try:
        with ThreadPoolExecutor(len(UNITS)) as ex:
            results = list(ex.map(compile_unit, range(len(UNITS))))
        for u, r in zip(UNITS, results):
            if verbose or r.returncode:
                print(r.stdout + r.stderr)
            if r.returncode:
                raise RuntimeError(f"nvcc failed on {u}")
        tmp = LIB_PATH + tag
        subprocess.run([nvcc()] + LINK_FLAGS + ["-o", tmp] + objs, check=True)
        os.replace(tmp, LIB_PATH)
    finally:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
    return LIB_PATH


if __name__ == "__main__":
    print(build_library(force=True, verbose=True))
