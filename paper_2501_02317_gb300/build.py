"""Builds libkhydro.so in-tree with nvcc for sm_103a (GB300).

The translation units are compiled in parallel and linked into one shared
library:
  * khy_fp64.cu    -- all-FP64 kernels, -fmad=false (bitwise-reproducible)
  * khy_mixed.cu   -- mixed-precision kernels (FP32 flux, FP64 state)
  * khy_single.cu  -- all-FP32 kernels (FP32 state and flux)
  * khy_runtime.cu -- C ABI, simulation objects, graphs, -fmad=false
  * khy_noalloc.cu -- the allocation-free one-step entry point
  * khy_batch.cu   -- many grids stepped together (batch engine)
  * khy_server.cu  -- serving loop with continuous batching

``python -m paper_2501_02317_gb300.build`` builds; ``build()`` is what
``__graft_entry__.build()`` calls.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from typing import List

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libkhydro.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fno-strict-aliasing",
          "-I" + os.path.join(ROOT, "include")]

UNITS = {
    "khy_fp64": ["-fmad=false"],
    "khy_mixed": [],
    "khy_single": [],
    "khy_runtime": ["-fmad=false"],
    "khy_noalloc": ["-fmad=false"],
    "khy_batch": ["-fmad=false"],
    "khy_server": ["-fmad=false"],
}


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libkhydro.so")


def _sources() -> List[str]:
    out = []
    for d in (CSRC, os.path.join(ROOT, "include")):
        for f in os.listdir(d):
            if f.endswith((".cu", ".cuh", ".h")):
                out.append(os.path.join(d, f))
    return out


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in _sources() + [os.path.abspath(__file__)])


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compiles and links libkhydro.so unless it is up to date."""
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    procs = []
    for unit, extra in UNITS.items():
        obj = os.path.join(BUILD, unit + ".o")
        cmd = [nvcc] + ARCH + COMMON + extra + (["-Xptxas", "-v"] if ptxas_info else []) + \
              ["-c", os.path.join(CSRC, unit + ".cu"), "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((unit, cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    logs = {}
    failed = []
    for unit, cmd, p in procs:
        out, _ = p.communicate()
        logs[unit] = out.decode(errors="replace")
        if p.returncode != 0:
            failed.append(unit)
    if failed:
        raise RuntimeError("nvcc failed for %s:\n%s" % (failed, "\n".join(logs[u] for u in failed)))
    if verbose or ptxas_info:
        for u in UNITS:
            if logs[u].strip():
                print(logs[u])
    tmp = LIB + ".tmp%d" % os.getpid()
    link = [nvcc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + \
           [os.path.join(BUILD, u + ".o") for u in UNITS] + \
           ["-Xlinker", "-rpath,/usr/local/cuda/lib64"]
    if verbose:
        print(" ".join(link), flush=True)
    subprocess.check_call(link)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv)
    print(LIB)
