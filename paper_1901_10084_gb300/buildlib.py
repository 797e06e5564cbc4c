"""Build the CUDA library libccdyk.so in-tree for sm_103a (nvcc, no cmake), and
its checked variant libccdyk_checked.so (CCD_CHECKED: the sweep kernels test
their offsets and report CC_ERR_BOUNDS instead of touching memory outside their
buffers).  Both compile in parallel."""
from __future__ import annotations

import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIBDIR = os.path.join(PKG, "_lib")
LIB = os.path.join(LIBDIR, "libccdyk.so")
LIB_CHECKED = os.path.join(LIBDIR, "libccdyk_checked.so")
SOURCES = [os.path.join(CSRC, "ccdyk.cu"), os.path.join(CSRC, "noalloc.cu")]
DEPENDS = SOURCES + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")] + [
    os.path.join(INCLUDE, "ccdyk.h")]

NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC", "-shared"]


def nvcc() -> str:
    for cand in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        p = os.path.join(cand, "bin", "nvcc") if cand else ""
        if p and os.path.exists(p):
            return p
    return "nvcc"


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(s) <= t for s in DEPENDS)


def build(force: bool = False, verbose: bool = False) -> str:
    """Build both libraries (only those out of date); returns the normal one."""
    os.makedirs(LIBDIR, exist_ok=True)
    jobs = []
    for lib, extra in ((LIB, []), (LIB_CHECKED, ["-DCCD_CHECKED"])):
        if not force and up_to_date(lib):
            continue
        tmp = lib + f".{os.getpid()}.tmp"
        cmd = [nvcc(), *NVCC_FLAGS, *extra, "-I" + INCLUDE, "-I" + CSRC, "-o", tmp, *SOURCES]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        jobs.append((subprocess.Popen(cmd), tmp, lib, cmd))
    for proc, tmp, lib, cmd in jobs:
        if proc.wait() != 0:
            raise subprocess.CalledProcessError(proc.returncode, cmd)
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
