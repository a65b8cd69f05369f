"""Build the solver library in-tree for sm_103a.

``python -m paper_1302_7193_gb300.build`` (or ``build()``) compiles
``csrc/pcg.cu`` into ``libpcg.so`` next to this file with nvcc.  There is
no other build system; the library has one translation unit.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libpcg.so")
SOURCES = [os.path.join(HERE, "csrc", "pcg.cu")]
DEPS = SOURCES + [os.path.join(HERE, "csrc", "kernels.cuh"), os.path.join(HERE, "csrc", "serve.cuh"),
                  os.path.join(HERE, "csrc", "multigrid.cuh"),
                  os.path.join(HERE, "csrc", "single_reduction.cuh"), os.path.join(HERE, "csrc", "serve_kernels.cuh"),
                  os.path.join(HERE, "csrc", "serve_mg.cuh"),
                  os.path.join(ROOT, "include", "pcg.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpcg.so")


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in DEPS)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    tmp = LIB + ".tmp"
    cmd = [nvcc_path(), "-shared", "-Xcompiler", "-fPIC", "-Xcompiler", "-pthread", *ARCH, "-O3", "-lineinfo", "-std=c++17",
           "-I", os.path.join(ROOT, "include"), "-o", tmp, *SOURCES]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
