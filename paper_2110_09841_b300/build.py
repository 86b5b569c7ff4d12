"""Build the CUDA library libkct.so (sm_103a) in-tree with nvcc."""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libkct.so")
SOURCES = [os.path.join(HERE, "csrc", "kct_api.cu")]
DEPS = [p for p in glob.glob(os.path.join(HERE, "csrc", "*")) if not p.endswith(("fp32_probe.cu", "conv3d_tc.cu"))] + \
    [os.path.join(ROOT, "include", "kct.h")]
# tensor-core 3D convolutions of the learned warm start
CONV_LIB = os.path.join(HERE, "libkct_conv.so")
CONV_SRC = os.path.join(HERE, "csrc", "conv3d_tc.cu")
CONV_DEPS = [CONV_SRC, os.path.join(ROOT, "include", "kct_conv.h"), os.path.join(ROOT, "include", "kct.h")]
# FP32 FMA throughput probe used by bench.py for the roofline denominator
PROBE_LIB = os.path.join(HERE, "libkct_probe.so")
PROBE_SRC = os.path.join(HERE, "csrc", "fp32_probe.cu")

NVCC_FLAGS = ["-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo",
              "-Xcompiler", "-fPIC", "-shared", "-Xptxas", "-warn-spills"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def stale(lib=LIB, deps=None) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in (DEPS + SOURCES if deps is None else deps))


def _compile(lib, sources, verbose):
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc(), *NVCC_FLAGS, "-I", os.path.join(ROOT, "include"), "-I", os.path.join(HERE, "csrc"),
           "-o", tmp, *sources]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)


def build(force: bool = False, verbose: bool = False) -> str:
    """Build libkct.so, the FP32 probe library and the convolution library if their sources
    changed."""
    if force or stale():
        _compile(LIB, SOURCES, verbose)
    if force or stale(PROBE_LIB, [PROBE_SRC]):
        _compile(PROBE_LIB, [PROBE_SRC], verbose)
    if force or stale(CONV_LIB, CONV_DEPS):
        _compile(CONV_LIB, [CONV_SRC], verbose)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
