"""Build the sm_103a CUDA library ``libhpmdr.so`` in-tree.

Each translation unit is compiled by nvcc in parallel for
``-gencode arch=compute_103a,code=sm_103a`` (no other target), then linked
into one shared library with the C ABI of ``include/hpmdr.h``.  No fast-math:
the kernels rely on IEEE round-to-nearest for the few floating-point steps.
"""
import concurrent.futures as cf
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libhpmdr.so")
UNITS = ["stats.cu", "decompose.cu", "lossless.cu", "select.cu", "recompose.cu", "qoi.cu", "cells.cu",
         "runtime.cu", "noalloc.cu", "serve.cu", "batch.cu", "gcells.cu", "bpdesign.cu"]
NVCC = os.environ.get("NVCC", "nvcc")
FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
         "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden", "-Xcompiler", "-ffp-contract=off", "-I", os.path.join(ROOT, "include")]


def _sources():
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(ROOT, "include", "hpmdr.h"))
    return deps


def _compile(unit):
    src = os.path.join(CSRC, unit)
    obj = os.path.join(OUT, unit + ".o")
    subprocess.run([NVCC, *FLAGS, "-c", src, "-o", obj], check=True)
    return obj


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= t for d in _sources()):
            return LIB
    os.makedirs(OUT, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(_compile, UNITS))
    tmp = LIB + ".tmp"
    subprocess.run([NVCC, "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-o", tmp,
                    *objs, "-lcudart"], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
