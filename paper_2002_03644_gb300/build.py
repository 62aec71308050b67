"""Build of libhlbm.so (the CUDA library behind include/hlbm.h) for sm_103a.

The translation units are compiled in parallel with nvcc into a private
folder, then linked into one shared object next to this file, which
``paper_2002_03644_gb300.hlbm`` loads.
"""
from __future__ import annotations

import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libhlbm.so")
# the debugging build: HLBM_DEBUG index checks in the step kernels (hlbm_debug_check)
LIB_DEBUG = os.path.join(PKG, "libhlbm_debug.so")
SOURCES = [os.path.join(CSRC, f) for f in ("hlbm_api.cu", "hlbm_noalloc.cu", "hlbm_surrogate.cu", "hlbm_selftest.cu")]
DEPS = SOURCES + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))] + [
    os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libhlbm")
    return exe


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in DEPS)


def build_library(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Build libhlbm.so, or with debug=True libhlbm_debug.so (the same
    sources with HLBM_DEBUG index checks)."""
    lib = LIB_DEBUG if debug else LIB
    if not force and up_to_date(lib):
        return lib
    tag = f"tmp{os.getpid()}{'d' if debug else ''}"
    objdir = os.path.join(PKG, "_build")
    os.makedirs(objdir, exist_ok=True)
    common = [nvcc(), "-O3", "-std=c++17", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC", "-I", INCLUDE]
    if debug:
        common.append("-DHLBM_DEBUG")
    if verbose:
        common.insert(1, "-Xptxas=-v")
    objs, procs = [], []
    for src in SOURCES:
        obj = os.path.join(objdir, os.path.basename(src)[:-3] + f".{tag}.o")
        objs.append(obj)
        procs.append(subprocess.Popen(common + ["-c", src, "-o", obj]))
    codes = [p.wait() for p in procs]
    if any(codes):
        raise subprocess.CalledProcessError(max(codes, key=abs), "nvcc")
    tmp = lib + f".{tag}"
    subprocess.run([nvcc(), *ARCH, "-shared", "-o", tmp, *objs], check=True)
    os.replace(tmp, lib)
    for o in objs:
        os.remove(o)
    return lib


if __name__ == "__main__":
    print(build_library(force=True, verbose=True))
