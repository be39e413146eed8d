"""Builds libfassmvs.so in-tree with nvcc for sm_103a (B300)."""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = sorted(glob.glob(os.path.join(HERE, "csrc", "*.cu")))
HDRS = sorted(glob.glob(os.path.join(HERE, "csrc", "*.cuh")) + glob.glob(os.path.join(HERE, "csrc", "*.h"))) + [
    os.path.join(os.path.dirname(HERE), "include", "fassmvs.h")]
LIB = os.path.join(HERE, "libfassmvs.so")
# the bounds-checked build (-DFASSMVS_CHECKED): every shared / global index the
# kernels form is tested first; a failure is recorded and the access skipped
LIB_CHECKED = os.path.join(HERE, "libfassmvs_checked.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo",
         "-Xcompiler", "-fPIC,-fvisibility=hidden", "-shared", "--expt-relaxed-constexpr",
         "-Xptxas", "-warn-spills"]


def stale(lib=LIB):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(f) > t for f in SRC + HDRS)


def build(force=False, verbose=False, checked=False):
    lib = LIB_CHECKED if checked else LIB
    if not force and not stale(lib):
        return lib
    cmd = [NVCC, *FLAGS, *(["-DFASSMVS_CHECKED"] if checked else []), "-o", lib, *SRC, "-lcudart"]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
        print(" ".join(cmd))
    subprocess.check_call(cmd)
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv, checked="--checked" in sys.argv)
    print(LIB_CHECKED if "--checked" in sys.argv else LIB)
