"""Build ``libtauleap.so`` (the engine's C ABI + sm_103a kernels) in-tree.

Each ``csrc/*.cu`` translation unit is compiled by nvcc for
``-gencode arch=compute_103a,code=sm_103a``; the FP64 reference kernels are
compiled with ``-fmad=false`` so that no multiply-add is contracted (their
results must equal the sequential IEEE statement of the algorithm bit for
bit).  The objects are linked into one shared library next to this file.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libtauleap.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2,-ffp-contract=off", "--expt-relaxed-constexpr",
          "-I", INCLUDE]
# per translation unit extra flags
UNITS = {
    "abi.cu": [],
    "kernel_warp_f64.cu": ["-fmad=false"],
    "kernel_lane_f64.cu": ["-fmad=false"],
    "kernel_lane_fast.cu": [],
    "server.cu": [],
    "moments.cu": [],
    "kernel_rre.cu": ["-fmad=false"],
    "peak.cu": ["-fmad=false"],
}


def nvcc() -> str:
    """Path of nvcc; the engine cannot be built without the CUDA toolkit."""
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libtauleap.so")
    return path


def _deps() -> list:
    out = []
    for d in (CSRC, INCLUDE):
        for f in os.listdir(d):
            if f.endswith((".cu", ".cuh", ".h")):
                out.append(os.path.join(d, f))
    return out


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every unit for sm_103a and link libtauleap.so in the package, unless it is newer than every source; returns its path."""
    newest = max(os.path.getmtime(p) for p in _deps() + [os.path.abspath(__file__)])
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    objs = []
    for unit, extra in UNITS.items():
        src = os.path.join(CSRC, unit)
        obj = os.path.join(BUILD, unit.replace(".cu", ".o"))
        cmd = [nvcc(), *ARCH, *COMMON, *extra, "-c", src, "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
            print(" ".join(cmd), flush=True)
        subprocess.run(cmd, check=True)
        objs.append(obj)
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.run([nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
