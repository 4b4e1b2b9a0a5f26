"""ORACLE (test infrastructure only): compile the plain-C oracle into oracle/liboracle_ugkwp.so.

Flags keep every floating-point operation an individual IEEE operation: no contraction into fused
multiply-adds, no fast-math reassociation (x86-64 SSE arithmetic has no excess precision).
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["oracle_rng.c", "oracle_math.c", "oracle_particles.c", "oracle_core.c"]
LIB = os.path.join(HERE, "liboracle_ugkwp.so")
CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", "-Wall",
          "-Wno-unused-function"]


def build(force: bool = False) -> str:
    deps = [os.path.join(HERE, s) for s in SOURCES] + [os.path.join(HERE, h) for h in
                                                       ("oracle.h", "oracle_internal.h", "oracle_particles.inc")]
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(os.path.getmtime(d) for d in deps):
        return LIB
    cmd = ["gcc", *CFLAGS, "-o", LIB + ".tmp", *[os.path.join(HERE, s) for s in SOURCES], "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
