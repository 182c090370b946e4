"""Builds the CUDA library libtm.so in-tree (nvcc, sm_103a only).

    python paper_2511_02036_gb300/build.py

Translation units are compiled in parallel; the link uses nvcc's static CUDA runtime so the
library needs nothing but the driver at run time.
"""

from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libtm.so")
# the bounds-checking variant (-DTM_DEBUG_BOUNDS): for tests, loaded through TM_LIBRARY
LIB_BOUNDS = os.path.join(PKG, "libtm_bounds.so")
SOURCES = ["kernels.cu", "runtime.cu", "server.cu", "culling.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -fmad=false and -ffp-contract=off: no contraction anywhere (device and host code), so every
# floating-point gate is the plain round-to-nearest evaluation of its stated expression.
NVCC_FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-fmad=false", "--prec-div=true",
              "--prec-sqrt=true", "-Xcompiler", "-fPIC,-ffp-contract=off,-O2",
              "-I" + INCLUDE, "-I" + CSRC]


def nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _stale(out, deps):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False, bounds=False):
    """Compiles the library (bounds=True: the bounds-checking variant, objects and library
    apart from the normal build's)."""
    out_dir = os.path.join(OUT_DIR, "bounds") if bounds else OUT_DIR
    lib = LIB_BOUNDS if bounds else LIB
    extra = ["-DTM_DEBUG_BOUNDS"] if bounds else []
    os.makedirs(out_dir, exist_ok=True)
    headers = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))]
    headers.append(os.path.join(INCLUDE, "tm.h"))
    objs, jobs = [], []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(out_dir, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + headers):
            jobs.append([nvcc(), *ARCH, *NVCC_FLAGS, *extra, "-c", s, "-o", o])

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        list(ex.map(run, jobs))
    if force or jobs or _stale(lib, objs):
        tmp = lib + ".tmp%d" % os.getpid()
        run([nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lpthread", "-ldl", "-lrt"])
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
