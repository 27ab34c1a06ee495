"""Compile the CUDA/C++ sources into the in-tree shared library libleafi.so.

nvcc targets sm_103a only (B300).  Host code is compiled with
-ffp-contract=off so the float64 tree statistics are evaluated exactly as
written (the kernels that must match them use explicit round-to-nearest
intrinsics).
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libleafi.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def sources():
    return sorted(glob.glob(os.path.join(HERE, "csrc", "*.cu")) +
                  glob.glob(os.path.join(HERE, "csrc", "*.cpp")))


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = sources() + glob.glob(os.path.join(HERE, "csrc", "*.h")) + \
        [os.path.join(ROOT, "include", "leafi.h")]
    return any(os.path.getmtime(p) > t for p in deps)


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [nvcc(), "-O3", "-std=c++17", ARCH, "-lineinfo", "-shared",
           "-Xcompiler", "-fPIC,-fopenmp,-ffp-contract=off",
           "-I", os.path.join(ROOT, "include"), "-o", tmp] + sources() + ["-lgomp"]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
        print(" ".join(cmd), file=sys.stderr)
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
