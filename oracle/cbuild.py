"""Compile the oracle's C parts (test infrastructure) with gcc: plain C,
-O2, OpenMP, no architecture-specific flags."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cproj.c")
LIB = os.path.join(HERE, "_cproj.so")


def build(force: bool = False) -> str:
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        subprocess.run(["gcc", "-O3", "-fopenmp", "-fPIC", "-shared", "-o", LIB, SRC, "-lm"], check=True)
    return LIB
