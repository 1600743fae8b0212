"""Build the CUDA library (libartsim.so) in-tree with nvcc for sm_103a.

One translation unit (csrc/sim_api.cu includes the kernels), compiled with
``-gencode arch=compute_103a,code=sm_103a``; the CUDA runtime is linked statically so the library
has no dependency beyond the driver.
"""
from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB_PATH = os.path.join(HERE, "libartsim.so")
SOURCES = [os.path.join(CSRC, f) for f in ("sim_api.cu", "step_kernel.cuh", "sim_internal.h")] + \
    [os.path.join(INCLUDE, "sim.h")]
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo", "-O3", "-std=c++17",
              "-Xcompiler", "-fPIC", "-shared", "-cudart", "static"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libartsim.so")


def build_library(force: bool = False, verbose: bool = False) -> str:
    stale = not os.path.exists(LIB_PATH) or any(os.path.getmtime(s) > os.path.getmtime(LIB_PATH) for s in SOURCES)
    if not (force or stale):
        return LIB_PATH
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = [nvcc()] + NVCC_FLAGS + (["-Xptxas", "-v"] if verbose else []) + \
        ["-o", tmp, os.path.join(CSRC, "sim_api.cu")]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    print(build_library(force=True, verbose=True))
