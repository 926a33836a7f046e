"""Builds libgs.so (the CUDA rasterizer behind include/gs.h) in-tree for sm_103a."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SOURCES = ["abi.cu", "preprocess.cu", "binning.cu", "composite.cu", "losses.cu", "appearance.cu", "static_scratch.cu",
           "peaks.cu"]
LIB = os.path.join(HERE, "libgs.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off,-O2",
         "-Xptxas", "-v", "--shared", "-I", os.path.join(ROOT, "include")]


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    srcs = [os.path.join(HERE, "csrc", s) for s in SOURCES]
    srcs += [os.path.join(HERE, "csrc", "gs_internal.cuh"), os.path.join(ROOT, "include", "gs.h"), __file__]
    return any(os.path.getmtime(s) > t for s in srcs)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not needs_build():
        return LIB
    nvcc = os.environ.get("NVCC", "nvcc")
    cmd = [nvcc, *ARCH, *FLAGS, "-o", LIB + ".tmp", *[os.path.join(HERE, "csrc", s) for s in SOURCES]]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("nvcc failed building libgs.so")
    if verbose:
        sys.stderr.write(r.stderr)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
    print(LIB)
