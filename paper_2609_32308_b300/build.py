"""Build libsd_b300.so in-tree for sm_103a (nvcc cross-compiles without a GPU)."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = [os.path.join(HERE, "csrc", f) for f in ("sd_kernels.cu", "sd_kernels_wide.cu", "sd_host.cpp", "sd_noalloc.cu", "sd_predictor.cu", "sd_peak.cu", "sd_sweep.cpp", "sd_synth.cpp")]
DEPS = SRC + [os.path.join(HERE, "csrc", "sd_internal.h"), os.path.join(ROOT, "include", "sd.h")]
LIB = os.path.join(HERE, "libsd_b300.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB) and all(
            os.path.getmtime(LIB) >= os.path.getmtime(p) for p in DEPS):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [NVCC, "-O3", "-std=c++17", "-lineinfo", *ARCH, "-shared", "-Xcompiler", "-fPIC",
           "-Xcompiler", "-O2", "-I", os.path.join(ROOT, "include"), "-o", tmp, *SRC]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
