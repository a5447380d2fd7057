"""Compile the oracle's C parts (test infrastructure) with gcc: plain C,
-O2, OpenMP, no architecture-specific flags."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, f) for f in ("cproj.c", "cscore.c")]
LIB = os.path.join(HERE, "_cproj.so")


def build(force: bool = False) -> str:
    if force or not os.path.exists(LIB) or any(os.path.getmtime(LIB) < os.path.getmtime(s) for s in SRCS):
        # -ffp-contract=off: one rounding per operation, as the definitions state
        subprocess.run(["gcc", "-O3", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-o", LIB, *SRCS, "-lm"],
                       check=True)
    return LIB
