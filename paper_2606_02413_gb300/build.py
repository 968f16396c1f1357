"""Builds librt.so in-tree with nvcc for sm_103a (GB300)."""
from __future__ import annotations

import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "librt.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def command(out=LIB, extra=()):
    cuda_lib = os.path.join(os.path.dirname(os.path.dirname(nvcc())), "lib64")
    # -ftz=true: single-precision denormals flush to zero.  No value of the
    # method comes near 1e-38 (the smallest are per-step optical depths of
    # ~1e-12), so results are bit-identical, and the reciprocal, square-root
    # and exponential intrinsics lose their denormal-range fix-ups.
    return ([nvcc()] + ARCH + ["-O3", "-ftz=true", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
                               "-cudart", "shared", f"-Xlinker=-rpath={cuda_lib}", "-I", INCLUDE, "-I", CSRC,
                               "-o", out] + list(extra) + sources())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every CUDA source into librt.so unless it is up to date."""
    if not force and os.path.exists(LIB):
        newest = max(os.path.getmtime(p) for p in _deps())
        if os.path.getmtime(LIB) >= newest:
            return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = command(tmp, ["-Xptxas", "-v"] if verbose else [])
    subprocess.check_call(cmd, cwd=ROOT)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose=True)
    print(LIB)
