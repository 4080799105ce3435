"""Builds libplasticarbor.so (the engine behind include/plastic_arbor.h) in-tree.

Every translation unit is compiled for sm_103a only.  The FP64 kernels and the
host builder are compiled without multiply-add contraction (--fmad=false,
-ffp-contract=off): the FP64 path is specified operation by operation.  The
mixed-precision and FP32-synapse kernels keep contraction on (their float-float
operations are written with explicitly rounded intrinsics).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libplasticarbor.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
          "-Xcompiler", "-Wall", "-Xptxas", "-warn-spills"]
NOFMA = ["--fmad=false", "-Xcompiler", "-ffp-contract=off"]

UNITS = {
    "step_fp64.cu": NOFMA,
    "step_mixed.cu": [],
    "step_fp32.cu": [],
    "events.cu": [],
    "model.cu": NOFMA,
    "epoch_noalloc.cu": NOFMA,
    "arith_check.cu": NOFMA,
    "fastforward.cu": NOFMA,
}


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found")
    return p


def _stale(out: str, deps) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


# the bounds-checked build (-DPA_CHECKED): every kernel index checked against
# its array, violations reported instead of performed; for the small parity
# cases, never for timing
CHECKED_LIB = os.path.join(HERE, "libplasticarbor_checked.so")


def build(force: bool = False, verbose: bool = False, ptxas_v: bool = False,
          checked: bool = False) -> str:
    if not checked:
        build(force, verbose, ptxas_v, checked=True)
    build_dir = os.path.join(BUILD, "checked") if checked else BUILD
    lib_path = CHECKED_LIB if checked else LIB
    extra = ["-DPA_CHECKED"] if checked else []
    os.makedirs(build_dir, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(INCLUDE, "plastic_arbor.h"))
    objs = []
    for unit, flags in UNITS.items():
        src = os.path.join(CSRC, unit)
        obj = os.path.join(build_dir, unit + ".o")
        objs.append(obj)
        if force or _stale(obj, [src, *headers, __file__]):
            cmd = [nvcc(), *ARCH, *COMMON, *flags, *extra, "-c", src, "-o", obj]
            if ptxas_v:
                cmd[1:1] = ["-Xptxas", "-v"]
            if verbose:
                print(" ".join(cmd))
            subprocess.check_call(cmd)
    if force or _stale(lib_path, objs):
        cmd = [nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", lib_path + ".tmp", *objs]
        if verbose:
            print(" ".join(cmd))
        subprocess.check_call(cmd)
        os.replace(lib_path + ".tmp", lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_v="-v" in sys.argv))
