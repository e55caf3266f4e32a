"""Writes atan_poly.cuh: the coefficients of the polynomial P with
atan(r) ~ r P(r^2) on r in [0, 1], used by the angle-storage tile's atan2
(octant reduction to |y|/|x| or |x|/|y| in [0, 1], then this polynomial).

Method: a degree-8 polynomial in s = r^2 fitted to atan(r)/r under the
weight r (so that the error is the absolute error of atan(r)) by Lawson's
iteratively reweighted least squares, which converges to the minimax
(Chebyshev) approximation, on 20001 Chebyshev-distributed points of [0, 1],
in FP64.  The approximation error is about 6e-9, far below the FP32 rounding
of the evaluation; the coefficients are stored rounded to FP32 (as hex
literals, so the header reproduces them exactly).

python paper_1211_0780_b300/csrc/atan_poly.py   (rewrites the header)
"""

from __future__ import annotations

import os

import numpy as np

DEGREE = 8
HEADER = os.path.join(os.path.dirname(os.path.abspath(__file__)), "atan_poly.cuh")


def fit(degree: int = DEGREE, points: int = 20001, iters: int = 80):
    """Coefficients c[0..degree] (increasing powers of s) and the maximum
    absolute error of r P(r^2) against atan(r) on the fitting points."""
    r = np.sort(0.5 + 0.5 * np.cos(np.linspace(0.0, np.pi, points)))
    s = r * r
    safe = np.where(r > 0, r, 1.0)
    f = np.where(r > 0, np.arctan(r) / safe, 1.0)
    V = np.vander(s, degree + 1, increasing=True)
    wt = np.full(points, 1.0 / points)
    c = None
    for _ in range(iters):
        sq = np.sqrt(wt)
        c = np.linalg.lstsq(V * (r * sq)[:, None], f * r * sq, rcond=None)[0]
        err = np.abs((V @ c - f) * r)
        wt = wt * err
        wt /= wt.sum()
    err = np.max(np.abs((V @ c - f) * r))
    return c, float(err)


def main() -> None:
    c, err = fit()
    c32 = c.astype(np.float32)
    lines = [
        "// Generated by atan_poly.py (do not edit): atan(r) ~ r P(r^2) on [0, 1],",
        f"// P of degree {DEGREE} in r^2, minimax under the weight r (Lawson's iteration,",
        f"// FP64); approximation error {err:.2e} before rounding the coefficients to FP32.",
        "#pragma once",
        "#include <cmath>",
        "",
        "namespace xy {",
        "",
        "// P(s) by Horner's rule with fused multiply-adds.",
        "__host__ __device__ __forceinline__ float atan_poly(float s) {",
        f"  float p = {float(c32[DEGREE]).hex()}f;  // s^{DEGREE}: {float(c32[DEGREE]):.9g}",
    ]
    for k in range(DEGREE - 1, -1, -1):
        v = float(c32[k])
        lines.append(f"  p = fmaf(p, s, {v.hex()}f);  // s^{k}: {v:.9g}")
    lines += ["  return p;", "}", ""]
    # the same polynomial for two values at once in the paired FP32
    # instructions of sm_100 and later (each lane rounds as fmaf does)
    lines += [
        "#ifdef __CUDACC__",
        "// P of two values at once (__ffma2_rn: each lane rounds as fmaf does).",
        "__device__ __forceinline__ float2 atan_poly2(float2 s) {",
        f"  float2 p = make_float2({float(c32[DEGREE]).hex()}f, {float(c32[DEGREE]).hex()}f);",
    ]
    for k in range(DEGREE - 1, -1, -1):
        v = float(c32[k]).hex()
        lines.append(f"  p = __ffma2_rn(p, s, make_float2({v}f, {v}f));")
    lines += ["  return p;", "}", "#endif", "", "}  // namespace xy", ""]
    with open(HEADER, "w") as fh:
        fh.write("\n".join(lines))
    print(HEADER, f"max |r P(r^2) - atan(r)| = {err:.3e}")


if __name__ == "__main__":
    main()
