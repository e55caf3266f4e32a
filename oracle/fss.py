"""FP64 oracle of the finite-size-scaling analysis -- TEST INFRASTRUCTURE.

Only ``tests/`` may import this module; the product path never calls it.
It follows Sec. II-III of the paper literally and shares no code with the
CUDA path:

* a resample is built as an explicit series: the bins of the original
  series (n_bins equal contiguous blocks, bin b = samples
  [b T / n_bins, (b + 1) T / n_bins)) repeated as often as the resample's
  multiplicity says, then reweighted like any series
  (:func:`oracle.reweight_observables`, exact at any beta');
* the crossing of two sizes' curves (Sec. III: rho_s L and U_L of different
  L intersect at T_c) is the root of A(beta') - B(beta') in the first grid
  interval where the difference changes sign, found with Brent's method on
  the exactly reweighted curves;
* the slopes there are the exact derivatives (fluctuation formula), and
  1/nu = ln(|slope_B| / |slope_A|) / ln(L_B / L_A) because a dimensionless
  ratio depends on t L^{1/nu} only (Sec. III, Eq. 7).
"""

from __future__ import annotations

import numpy as np
from scipy.optimize import brentq

from . import reweight_observables


def bin_edges(T: int, n_bins: int) -> np.ndarray:
    return np.array([T * b // n_bins for b in range(n_bins + 1)], dtype=np.int64)


def resampled_series(series: dict, n_bins: int, counts_row) -> dict:
    """The series of one resample: bin b repeated counts_row[b] times, bins
    in order.  Columns as in the product's series dict (c, s2 of shape
    (3, T))."""
    T = len(series["E"])
    edges = bin_edges(T, n_bins)
    idx = np.concatenate([np.tile(np.arange(edges[b], edges[b + 1]), int(n)) for b, n in enumerate(counts_row)])
    return {"E": np.asarray(series["E"], np.float64)[idx],
            "m2": np.asarray(series["m2"], np.float64)[idx],
            "m4": np.asarray(series["m4"], np.float64)[idx],
            "c": np.asarray(series["c"], np.float64)[:, idx],
            "s2": np.asarray(series["s2"], np.float64)[:, idx]}


def curves_at(series: dict, beta0: float, betap, L: int) -> dict:
    """U_L, rho_s L and their derivatives at each beta' (exact reweighting)."""
    return reweight_observables(series["E"], series["m2"], series["m4"], np.asarray(series["c"]).T,
                                np.asarray(series["s2"]).T, beta0, np.atleast_1d(betap), L)


def crossing_of(fA, dfA, fB, dfB, grid, LA: float, LB: float):
    """Crossing of two curves given as callables of beta' (value and
    derivative): first grid interval with a sign change of fA - fB, root by
    Brent's method, slopes there, 1/nu from their ratio.  Returns
    (beta*, slopeA, slopeB, 1/nu, nu) or NaNs."""
    g = np.array([fA(b) - fB(b) for b in grid])
    for k in range(len(grid) - 1):
        if not (np.isfinite(g[k]) and np.isfinite(g[k + 1])):
            continue
        if g[k] == 0.0:
            root = grid[k]
        elif g[k + 1] != 0.0 and (g[k] < 0.0) != (g[k + 1] < 0.0):
            root = brentq(lambda b: fA(b) - fB(b), grid[k], grid[k + 1], xtol=1e-15, rtol=1e-15, maxiter=200)
        else:
            continue
        sA, sB = dfA(root), dfB(root)
        inv_nu = np.log(abs(sB) / abs(sA)) / np.log(LB / LA)
        return root, sA, sB, inv_nu, 1.0 / inv_nu
    nan = float("nan")
    return nan, nan, nan, nan, nan


def crossing(seriesA: dict, LA: int, seriesB: dict, LB: int, beta0: float, grid, which: str = "U"):
    """Crossing of the exactly reweighted curves of two series."""
    key, dkey = (("U", "dU") if which == "U" else ("rhoL", "drhoL"))

    def f(s, L, k):
        return lambda b: float(curves_at(s, beta0, [b], L)[k][0])

    return crossing_of(f(seriesA, LA, key), f(seriesA, LA, dkey), f(seriesB, LB, key), f(seriesB, LB, dkey),
                       np.asarray(grid, np.float64), float(LA), float(LB))
