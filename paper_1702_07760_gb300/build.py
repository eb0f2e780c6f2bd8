"""Builds the CUDA library libsph.so in-tree for sm_103a with nvcc.

Each translation unit is compiled to an object in parallel (under _build/),
then linked into one shared library."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libsph.so")
# the bounds-checked variant (-DSPH_CHECKED), for debugging and its tests
LIB_CHECKED = os.path.join(HERE, "libsph_checked.so")
OBJ_DIR = os.path.join(ROOT, "_build")
SOURCES = ["sph_api.cu", "sph_noalloc.cu", "mpnn.cu", "fma_peak.cu"]
HEADERS = ["sph_kernels.cuh", "umma.cuh"]
PUBLIC_HEADERS = ["sph.h", "sph_surrogate.h"]
FLAGS = ["-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo", "-Xcompiler", "-fPIC"]


def _includes():
    return ["-I", os.path.join(ROOT, "include"), "-I", CSRC]


def nvcc_command(out: str = LIB, extra=()):
    """One nvcc invocation compiling and linking every source (used to inspect
    ptxas output)."""
    return ["nvcc", *FLAGS, "-shared", *_includes(), *extra, "-o", out,
            *[os.path.join(CSRC, s) for s in SOURCES]]


def stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + \
        [os.path.join(ROOT, "include", h) for h in PUBLIC_HEADERS]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compiles libsph.so (or, with checked, libsph_checked.so with every index
    read from device data tested) and returns its path."""
    lib = LIB_CHECKED if checked else LIB
    if not (force or stale(lib)):
        return lib
    os.makedirs(OBJ_DIR, exist_ok=True)
    extra = ["-Xptxas", "-v"] if verbose else []
    if checked:
        extra += ["-DSPH_CHECKED"]
    procs, objs = [], []
    for s in SOURCES:
        obj = os.path.join(OBJ_DIR, os.path.splitext(s)[0] + f"{'.checked' if checked else ''}.{os.getpid()}.o")
        objs.append(obj)
        procs.append(subprocess.Popen(["nvcc", *FLAGS, *_includes(), *extra, "-c", "-o", obj,
                                       os.path.join(CSRC, s)]))
    codes = [p.wait() for p in procs]
    if any(codes):
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
        raise subprocess.CalledProcessError(max(codes, key=abs), "nvcc")
    tmp = lib + f".tmp{os.getpid()}"
    subprocess.check_call(["nvcc", "-shared", "-gencode", "arch=compute_103a,code=sm_103a", "-o", tmp, *objs])
    for o in objs:
        os.remove(o)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
