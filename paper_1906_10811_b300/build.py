"""Build the CUDA library libfd_b300.so in-tree with nvcc for sm_103a."""

import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libfd_b300.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


def sources():
    return sorted(glob.glob(os.path.join(HERE, "csrc", "*.cu")) +
                  glob.glob(os.path.join(HERE, "csrc", "*.cuh")) +
                  [os.path.join(ROOT, "include", "fd.h")])


def command(out=LIB, extra=()):
    return [NVCC, "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo", "-O3", "-std=c++17",
            "-Xcompiler", "-fPIC", "-shared", "-cudart", "shared",
            "-Xlinker", "-rpath,/usr/local/cuda/lib64", *extra,
            "-o", out, os.path.join(HERE, "csrc", "fd_capi.cu")]


def build(force=False, verbose=False):
    """Compile if any source is newer than the library; returns the library path."""
    if not force and os.path.exists(LIB):
        newest = max(os.path.getmtime(s) for s in sources())
        if os.path.getmtime(LIB) >= newest:
            return LIB
    cmd = command()
    if verbose:
        print(" ".join(cmd))
    subprocess.check_call(cmd)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose=True)
