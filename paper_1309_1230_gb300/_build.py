"""Builds the CUDA library ``libswe.so`` in-tree for sm_103a with nvcc.

Each translation unit under ``csrc/`` is compiled in parallel, then linked
into one shared library exporting the C ABI of ``include/swe.h``.  The
library is rebuilt when any source or header is newer than it.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libswe.so")
# The checked build (-DSWE_CHECKED): device-side index and alignment checks in
# the fused and batched row steps that record a failure in the step flags and
# skip the access, and NaN in every byte of the planes' padding; for tests.
CHECKED_DIR = os.path.join(OUT_DIR, "checked")
LIB_CHECKED = os.path.join(CHECKED_DIR, "libswe_checked.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# FP32 arithmetic uses approximate division/square root with flush-to-zero
# (these flags do not touch FP64, which stays IEEE).  No implicit multiply-add
# contraction: the kernels write their FMAs out, so every kernel form rounds a
# cell identically.
NVFLAGS = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2",
                  "-ftz=true", "-prec-div=false", "-prec-sqrt=false", "-fmad=false",
                  "-I", INCLUDE]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h")) + [
        os.path.abspath(__file__)]


def up_to_date(checked: bool = False) -> bool:
    lib = LIB_CHECKED if checked else LIB
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False, checked: bool = False) -> str:
    lib = LIB_CHECKED if checked else LIB
    out_dir = CHECKED_DIR if checked else OUT_DIR
    if not force and up_to_date(checked):
        return lib
    os.makedirs(out_dir, exist_ok=True)
    srcs = sources()
    objs = [os.path.join(out_dir, os.path.basename(s)[:-3] + ".o") for s in srcs]
    extra = (["-Xptxas", "-v"] if ptxas_info else []) + (["-DSWE_CHECKED"] if checked else [])

    def comp(pair):
        src, obj = pair
        cmd = [nvcc()] + NVFLAGS + extra + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        return src, r

    with ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        results = list(ex.map(comp, zip(srcs, objs)))
    failed = [(s, r) for s, r in results if r.returncode != 0]
    for s, r in results:
        if verbose or ptxas_info or r.returncode != 0:
            sys.stderr.write(f"== {os.path.basename(s)}\n{r.stdout}{r.stderr}")
    if failed:
        raise RuntimeError("nvcc failed on: " + ", ".join(os.path.basename(s) for s, _ in failed))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
