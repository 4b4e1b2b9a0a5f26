"""Compile libugkwp.so (the CUDA kernels and the C ABI of include/ugkwp.h) in-tree for sm_103a.

ugkwp_core.cu (which includes the wave fluxes, ugkwp_flux.cuh) is compiled with -fmad=false so that every
floating-point operation of the step is an individually rounded IEEE operation (fused multiply-adds only where
the code asks for them), the same in the step's kernels and in the batched persistent kernel.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libugkwp.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off", "-I", os.path.join(ROOT, "include")]
UNITS = {"ugkwp_core.cu": ["-fmad=false"], "ugkwp_mlp.cu": []}
DEPS = ["ugkwp_internal.h", "ugkwp_detmath.cuh", "ugkwp_flux.cuh"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    srcs = [os.path.join(CSRC, u) for u in UNITS] + [os.path.join(CSRC, d) for d in DEPS]
    srcs.append(os.path.join(ROOT, "include", "ugkwp.h"))
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(os.path.getmtime(s) for s in srcs):
        return LIB
    bdir = os.path.join(HERE, "_build")
    os.makedirs(bdir, exist_ok=True)
    objs = []
    for unit, flags in UNITS.items():
        obj = os.path.join(bdir, unit.replace(".cu", ".o"))
        cmd = [_nvcc(), *ARCH, *COMMON, *flags, "-c", os.path.join(CSRC, unit), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        subprocess.run(cmd, check=True)
        objs.append(obj)
    tmp = LIB + ".tmp"
    subprocess.run([_nvcc(), *ARCH, "-shared", "-o", tmp, *objs], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
