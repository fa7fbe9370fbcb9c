"""Build the sm_103a CUDA library ``_lib/libtlsph.so`` in-tree with nvcc."""
from __future__ import annotations

import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "_lib", "libtlsph.so")
DEBUG_LIB = os.path.join(HERE, "_lib", "libtlsph_debug.so")  # with device bounds checks (TLSPH_DEBUG)
SOURCES = [os.path.join(HERE, "csrc", "tlsph_capi.cu")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _inputs():
    return glob.glob(os.path.join(HERE, "csrc", "*")) + [os.path.join(ROOT, "include", "tlsph.h")]


def nvcc_command(out: str = LIB, extra=()):
    # --fmad=false: no implicit multiply-add contraction, so a kernel's rounding does not depend
    # on the code around it (execution modes and block sizes give bit-identical steps); the hot
    # loops write their fused multiply-adds explicitly.
    # --split-compile 0: the device code's optimisation passes run on all host cores
    return (["nvcc", "-std=c++17", "-O3", *ARCH, "-lineinfo", "--fmad=false", "-Xcompiler", "-fPIC",
             "-Xcompiler", "-ffp-contract=off", "--split-compile", "0", "-shared", "-o", out, *SOURCES]
            + list(extra))


def build_library(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Compile if the library is missing or older than any source; return its path.  debug=True builds
    libtlsph_debug.so, whose kernels check every neighbour index (a bad one sets a flag that the step
    reports as a status; nothing traps)."""
    lib = DEBUG_LIB if debug else LIB
    os.makedirs(os.path.dirname(lib), exist_ok=True)
    if not force and os.path.exists(lib):
        t = os.path.getmtime(lib)
        if all(os.path.getmtime(p) <= t for p in _inputs()):
            return lib
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = nvcc_command(tmp, ["-DTLSPH_DEBUG"] if debug else [])
    if verbose:
        print(" ".join(cmd))
    subprocess.check_call(cmd)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build_library(force=True, verbose=True))
