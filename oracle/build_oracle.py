"""Compiles the FP64 CPU oracle (test infrastructure) into oracle/libpa_oracle.so.

Built without floating-point contraction so that every a*b+c in pa_oracle.c is
two roundings unless it is written as fma(); this is the arithmetic the CUDA
engine's FP64 path reproduces.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "libpa_oracle.so")


def build(force: bool = False) -> str:
    src = os.path.join(HERE, "pa_oracle.c")
    hdr = os.path.join(HERE, "pa_oracle.h")
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return LIB
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-fopenmp", "-Wall", "-Wno-unused-function",
           "-o", LIB + ".tmp", src, "-lm"]
    subprocess.check_call(cmd)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
