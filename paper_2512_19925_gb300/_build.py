"""Compile the CUDA library in-tree for sm_103a (GB300).

Each translation unit is compiled on its own (in parallel) and linked into
``_build/libhww.so`` with the CUDA runtime linked statically.  Translation
units are built with contraction off (``-fmad=false`` on the device,
``-ffp-contract=off`` on the host): the FP64 units because their arithmetic
is part of the numerics contract with the CPU oracle, the FP32 tracking unit
so that the single-problem and batched kernels, which inline the same event
loop, round every expression the same way (its fused multiply-adds are
written out as fmaf).
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libhww.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
          "-I" + INCLUDE, "-I" + CSRC]
UNITS = {
    "api.cu": ["-fmad=false"],
    "step.cu": ["-fmad=false"],
    "losm.cu": ["-fmad=false"],
    "noalloc.cu": ["-fmad=false"],
    "measure.cu": [],
    "track_fp64.cu": ["-fmad=false"],
    "track_fp32.cu": ["-fmad=false"],
}


def nvcc() -> str:
    path = shutil.which("nvcc")
    if path:
        return path
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def _sources():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".inc"))] + [
        os.path.join(INCLUDE, "hww.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    """Build the library if a source is newer than it; returns its path."""
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    objs = []

    def compile_one(name):
        obj = os.path.join(BUILD, name.replace(".cu", ".o"))
        cmd = [cc] + ARCH + COMMON + UNITS[name] + ["-c", os.path.join(CSRC, name), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (name, " ".join(cmd), r.stderr))
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(compile_one, sorted(UNITS)))
    tmp = LIB + ".%d.tmp" % os.getpid()
    cmd = [cc] + ARCH + ["-shared", "-Xlinker", "--no-undefined", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
