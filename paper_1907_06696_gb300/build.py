"""Build the CUDA library libstokes_gb300.so in-tree for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked into one
shared library next to this file. No CMake, no torch extension machinery.
build(debug=True) links libstokes_gb300_debug.so: the translation units that
STOKES_DEBUG changes (the octree kernels' index-map checks and the status
reads of the C ABI) compiled with it, the others shared with the release build.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libstokes_gb300.so")
DEBUG_LIB = os.path.join(HERE, "libstokes_gb300_debug.so")
SOURCES = ["ops.cu", "vec.cu", "krylov.cu", "brick.cu", "brick_tc.cu", "batch.cu", "outer.cu", "outer_tc.cu", "octree.cu",
           "octree_host.cpp", "api.cu", "noalloc.cu", "probe.cu"]
DEBUG_SOURCES = ["octree.cu", "api.cu"]   # the only sources that test STOKES_DEBUG
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC,-ffp-contract=off",
         "-I" + os.path.join(ROOT, "include")]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libstokes_gb300.so")
    return cand


def _stale(obj: str, deps) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, force: bool = False, debug: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(ROOT, "include", "stokes.h"))
    cc = nvcc()

    def compile_one(src):
        dbg = debug and src in DEBUG_SOURCES
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, os.path.splitext(src)[0] + ("_debug.o" if dbg else ".o"))
        if force or _stale(o, [s] + headers):
            cmd = [cc] + ARCH + FLAGS + (["-DSTOKES_DEBUG"] if dbg else []) + ["-c", s, "-o", o]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
            if verbose and r.stderr:
                print(r.stderr)
        return o

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    lib = DEBUG_LIB if debug else LIB
    if force or _stale(lib, objs):
        cmd = [cc] + ARCH + ["-shared", "-o", lib] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    return lib


if __name__ == "__main__":
    print(build(verbose=True))
