"""Builds libgscl.so in-tree with nvcc for sm_103a (cross-compiles without a GPU).

The CUDA runtime is linked statically and the driver is reached at run time
through the runtime's entry-point query, so the library loads on a machine
without a GPU driver (its calls then fail with GSCL_ERR_CUDA).
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libgscl.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

NVCC_FLAGS = [
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-O3", "-lineinfo", "-std=c++17",
    "-Xcompiler", "-fPIC,-O2",
]
OBJ_DIR = os.path.join(HERE, "_build")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def deps():
    return (sources() + sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")))
            + [os.path.join(INCLUDE, "gscl.h")])


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in deps())


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    """Compiles every .cu under csrc/ (in parallel) into one shared library next to this file."""
    if not force and not needs_build():
        return LIB
    nvcc = os.environ.get("NVCC", "nvcc")
    os.makedirs(OBJ_DIR, exist_ok=True)
    tag = os.getpid()

    def compile_one(src):
        obj = os.path.join(OBJ_DIR, os.path.basename(src)[:-3] + f".{tag}.o")
        cmd = [nvcc, *NVCC_FLAGS, *extra, "-I", INCLUDE, "-c", "-o", obj, src]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        out = subprocess.run(cmd, capture_output=True, text=True)
        if out.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{out.stderr}")
        if verbose and out.stderr:
            print(out.stderr, file=sys.stderr)
        return obj

    srcs = sources()
    objs = [os.path.join(OBJ_DIR, os.path.basename(s)[:-3] + f".{tag}.o") for s in srcs]
    tmp = LIB + f".tmp{tag}"
    try:
        with ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 1))) as ex:
            list(ex.map(compile_one, srcs))
        subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-cudart", "static",
                               "-o", tmp, *objs])
        os.replace(tmp, LIB)
    finally:  # no objects left behind, whether or not a step failed
        for o in objs + [tmp]:
            if os.path.exists(o):
                os.remove(o)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra=["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else [])
    print(LIB)
