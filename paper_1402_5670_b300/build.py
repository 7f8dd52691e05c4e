"""Build libshearlet.so in-tree with nvcc for sm_103a (B300).

    python -m paper_1402_5670_b300.build [--verbose]

The shared library lands next to this file; the ctypes binding loads it from there.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libshearlet.so")
SOURCES = ["shearlet.cu", "bank_host.cpp", "mlp.cu"]
HEADERS = ["fft_core.cuh", "kernels2d.cuh", "kernels3d.cuh", "kernels_cluster.cuh", "kernels_tc.cuh",
           "kernels_roww.cuh",
           "bank_host.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _inputs():
    return ([os.path.join(CSRC, s) for s in SOURCES + HEADERS]
            + [os.path.join(ROOT, "include", "shearlet.h"), os.path.abspath(__file__)])


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in _inputs())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every source to an object (the sources in parallel), then link the
    shared library."""
    if not force and up_to_date():
        return LIB
    obj_dir = os.path.join(HERE, "_build")
    os.makedirs(obj_dir, exist_ok=True)
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC,-O3", *ARCH, "-lineinfo",
              "-I", os.path.join(ROOT, "include")]
    if verbose:
        common.insert(0, "-Xptxas=-v")
    procs, objs = [], []
    for src in SOURCES:
        obj = os.path.join(obj_dir, os.path.splitext(src)[0] + ".o")
        # no split compilation for the transform kernels: their device code is then the
        # same whatever the build host, and measured fastest; the MLP file is split
        extra = ["--split-compile=8"] if src == "mlp.cu" else []
        cmd = [nvcc(), *common, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append(subprocess.Popen(cmd))
        objs.append(obj)
    failed = [p.args for p in procs if p.wait() != 0]
    if failed:
        raise subprocess.CalledProcessError(1, failed[0])
    link = [nvcc(), "-shared", *ARCH, "-o", LIB + ".tmp", *objs, "-lpthread"]
    subprocess.run(link, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose="--verbose" in sys.argv)
    print(LIB)
