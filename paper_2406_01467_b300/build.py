"""Builds libgs.so (the CUDA rasterizer behind include/gs.h) in-tree for sm_103a,
and on request libgs_debug.so, the same sources with -DGS_DEBUG (device-side
bounds checks of the data-dependent indices; a test harness, not the product)."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SOURCES = ["abi.cu", "preprocess.cu", "binning.cu", "composite.cu", "losses.cu", "appearance.cu", "static_scratch.cu",
           "peaks.cu"]
LIB = os.path.join(HERE, "libgs.so")
DEBUG_LIB = os.path.join(HERE, "libgs_debug.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off,-O2",
         "-Xptxas", "-v", "--shared", "-I", os.path.join(ROOT, "include")]


def needs_build(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    srcs = [os.path.join(HERE, "csrc", s) for s in SOURCES]
    srcs += [os.path.join(HERE, "csrc", "gs_internal.cuh"), os.path.join(ROOT, "include", "gs.h"), __file__]
    return any(os.path.getmtime(s) > t for s in srcs)


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    lib = DEBUG_LIB if debug else LIB
    if not force and not needs_build(lib):
        return lib
    nvcc = os.environ.get("NVCC", "nvcc")
    extra = ["-DGS_DEBUG"] if debug else []
    cmd = [nvcc, *ARCH, *FLAGS, *extra, "-o", lib + ".tmp", *[os.path.join(HERE, "csrc", s) for s in SOURCES]]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError(f"nvcc failed building {os.path.basename(lib)}")
    if verbose:
        sys.stderr.write(r.stderr)
    os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, debug="--debug" in sys.argv))
