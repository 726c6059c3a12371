"""Build the CUDA library libeot.so (sm_103a) in-tree with nvcc.

Each translation unit of ``csrc/`` is compiled in parallel, then linked into
``_lib/libeot.so`` with the CUDA runtime linked statically.  Run as a module
(``python -m paper_2506_14780_gb300.build``) or call ``build()``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_lib")
OBJ_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libeot.so")
# the bounds-checked build (-DEOT_DEBUG): its own objects and library
OBJ_DIR_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(OUT_DIR, "libeot_debug.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + INCLUDE,
          "-diag-suppress", "550"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libeot.so")
    return cand


def sources() -> list:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _compile(src: str, verbose: bool, debug: bool = False) -> str:
    obj = os.path.join(OBJ_DIR_DEBUG if debug else OBJ_DIR, os.path.basename(src)[:-3] + ".o")
    if os.path.exists(obj):
        newest = max(os.path.getmtime(p) for p in
                     [src] + [os.path.join(CSRC, h) for h in os.listdir(CSRC)
                              if h.endswith((".h", ".cuh"))] + [os.path.join(INCLUDE, "eot.h")])
        if os.path.getmtime(obj) >= newest:
            return obj
    cmd = [_nvcc()] + CFLAGS + (["-DEOT_DEBUG"] if debug else []) + ARCH + ["-c", src, "-o", obj]
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def build(verbose: bool = False, debug: bool = False) -> str:
    """Compile and link; returns the path of libeot.so (debug: libeot_debug.so,
    the kernels' bounds checks compiled in, see eot_debug_build)."""
    lib = LIB_DEBUG if debug else LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    os.makedirs(OBJ_DIR_DEBUG if debug else OBJ_DIR, exist_ok=True)
    srcs = sources()
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose, debug), srcs))
    tmp = lib + ".tmp"
    # -ldl: the NVTX v3 header finds a profiler's injection library with dlopen
    cmd = [_nvcc(), "-shared"] + ARCH + ["-o", tmp] + objs + ["-ldl"]
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, debug="--debug" in sys.argv))
