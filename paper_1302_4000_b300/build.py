"""Build libclusco.so in-tree with nvcc for sm_103a (B300).

``python -m paper_1302_4000_b300.build`` (or ``build()``) compiles the unity source
``csrc/clusco.cu`` into ``paper_1302_4000_b300/libclusco.so``. The library links only the
CUDA runtime (static) and resolves the driver entry point it needs for TMA descriptors at
run time, so the same .so cross-compiles here and runs on the GPU machine.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc", "clusco.cu")
LIB = os.path.join(HERE, "libclusco.so")
# the test-hook build (include/clusco_debug.h): same sources, hooks compiled in, 0.2 s device waits
DEBUG_LIB = os.path.join(HERE, "libclusco_debug.so")
DEBUG_FLAGS = ("-DCLUSCO_DEBUG_HOOKS", "-DCLUSCO_WAIT_NS=200000000ull")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return [SRC] + sorted(glob.glob(os.path.join(HERE, "csrc", "*.cuh"))) + sorted(
        glob.glob(os.path.join(os.path.dirname(HERE), "include", "*.h")))


def stale(out: str = LIB) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(s) > t for s in sources())


def build(out: str = LIB, extra=(), verbose: bool = False, force: bool = False) -> str:
    if not force and not stale(out) and (not extra or out == DEBUG_LIB):
        return out
    nvcc = os.environ.get("NVCC", "nvcc")
    cmd = [nvcc, *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
           "--expt-relaxed-constexpr", *extra, SRC, "-o", out]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError(f"nvcc failed ({r.returncode}) building {out}")
    if verbose:
        sys.stderr.write(r.stderr)
    return out


def build_debug(force: bool = False) -> str:
    """The test-hook library (never loaded by the package itself)."""
    return build(DEBUG_LIB, extra=DEBUG_FLAGS, force=force)


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force=True))
