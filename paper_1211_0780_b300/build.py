"""Builds the in-tree CUDA library ``libxy.so`` for sm_103a (B300), and its
bounds-checked debug twin ``libxy_check.so`` (compiled with XY_BOUNDS_CHECK:
every spin access of the sweep kernels is checked against its slot and a
stray one is skipped and reported as XY_ERR_BOUNDS instead of faulting; it
stands in for compute-sanitizer, which this project cannot rely on).

``python -m paper_1211_0780_b300.build [--force] [--no-check]`` or
:func:`build`.  nvcc cross-compiles without a GPU; the shared objects land
next to this file so that they travel with the source tree.
"""

from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
SOURCES = ["libxy.cu", "reweight.cu", "fss.cu", "multihist.cu", "peaks.cu", "ladder.cpp"]
HEADERS = ["philox.cuh", "sweep.cuh", "kernels.cuh", "persistent.cuh", "atan_poly.cuh"]
LIB = os.path.join(HERE, "libxy.so")
CHECK_LIB = os.path.join(HERE, "libxy_check.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-shared", "-Xcompiler", "-fPIC,-O2",
         "-Xptxas", "-v"]


def _inputs():
    srcs = [os.path.join(CSRC, s) for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]
    deps = srcs + [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "xy.h")]
    return srcs, [d for d in deps if os.path.exists(d)]


def needs_build(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(d) > t for d in _inputs()[1])


def _compile(lib: str, extra: list[str], verbose: bool) -> None:
    srcs, _ = _inputs()
    nvcc = os.environ.get("NVCC", "nvcc")
    res = subprocess.run([nvcc, *ARCH, *FLAGS, *extra, "-o", lib, *srcs], capture_output=True, text=True)
    if verbose or res.returncode != 0:
        sys.stderr.write(res.stdout + res.stderr)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed building {os.path.basename(lib)}")


def build(force: bool = False, verbose: bool = False, check: bool = True) -> str:
    """Builds libxy.so (and libxy_check.so unless check=False) when a source
    is newer or `force`; the two compile in parallel.  Returns LIB."""
    jobs = [(LIB, [])]
    if check:
        jobs.append((CHECK_LIB, ["-DXY_BOUNDS_CHECK"]))
    jobs = [(lib, extra) for lib, extra in jobs if force or needs_build(lib)]
    with ThreadPoolExecutor(max_workers=2) as ex:
        for f in [ex.submit(_compile, lib, extra, verbose) for lib, extra in jobs]:
            f.result()
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, check="--no-check" not in sys.argv)
    print(LIB)
