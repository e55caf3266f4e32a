"""Builds the in-tree CUDA library ``libxy.so`` for sm_103a (B300).

``python -m paper_1211_0780_b300.build`` or :func:`build`.  nvcc
cross-compiles without a GPU; the shared object lands next to this file so
that it travels with the source tree.
"""

from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
SOURCES = ["libxy.cu", "reweight.cu", "fss.cu", "multihist.cu", "peaks.cu", "ladder.cpp"]
HEADERS = ["philox.cuh", "sweep.cuh", "kernels.cuh", "persistent.cuh"]
LIB = os.path.join(HERE, "libxy.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-shared", "-Xcompiler", "-fPIC,-O2",
         "-Xptxas", "-v"]


def _inputs():
    srcs = [os.path.join(CSRC, s) for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]
    deps = srcs + [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "xy.h")]
    return srcs, [d for d in deps if os.path.exists(d)]


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(d) > t for d in _inputs()[1])


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not needs_build():
        return LIB
    srcs, _ = _inputs()
    nvcc = os.environ.get("NVCC", "nvcc")
    cmd = [nvcc, *ARCH, *FLAGS, "-o", LIB, *srcs]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if verbose or res.returncode != 0:
        sys.stderr.write(res.stdout + res.stderr)
    if res.returncode != 0:
        raise RuntimeError("nvcc failed building libxy.so")
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
    print(LIB)
