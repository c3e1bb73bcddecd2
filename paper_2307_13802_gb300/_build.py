"""Compiles the CUDA library ``libsusp.so`` in-tree for sm_103a.

Translation units are compiled in parallel with nvcc and linked as one shared
library with the CUDA runtime linked statically.  The double-precision
integrator, neighbour build and utilities are compiled without multiply-add
contraction (``-fmad=false``) so that their sums and products round as
written (the list's cutoff decisions and the state updates then repeat the
oracle's bit for bit); the FP64 pair kernel and the mixed-precision kernels
use contraction.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libsusp.so")
BUILD = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
          "-Xcompiler", "-ffp-contract=off"]
# (source, extra flags)
UNITS = [
    ("api.cu", []),
    ("k_pair_fp64.cu", ["-fmad=true"]),
    ("k_integrate_fp64.cu", ["-fmad=false"]),
    ("k_neighbors.cu", ["-fmad=false"]),
    ("k_util.cu", ["-fmad=false"]),
    ("k_mixed.cu", ["-fmad=true"]),
    ("k_pair_mixed.cu", ["-fmad=true", "-prec-div=false", "-prec-sqrt=false"]),
    ("noalloc.cu", ["-fmad=false"]),
    ("k_det.cu", ["-fmad=false"]),
]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsusp.so")


def _sources_newer_than(target: str) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(HERE, "..", "include", "susp.h"))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    if not force and not _sources_newer_than(LIB):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()

    def compile_one(unit):
        src, flags = unit
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *COMMON, *flags, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(compile_one, UNITS))
    tmp = LIB + ".tmp"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True))
