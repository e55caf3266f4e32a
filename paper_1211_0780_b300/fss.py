"""Finite-size-scaling analysis on the device (Sec. III of the paper).

The measured series of each lattice size is binned (the paper blocks its
measurements into bins before any analysis, Sec. II), reweighted bin by bin
to a grid of couplings (``xy_reweight_bins``), and resampled by whole bins
(bootstrap with replacement, or jackknife): every resample's reweighted
curves of the Binder cumulant U_L (Eq. 5) and of rho_s L (Eq. 6) with their
beta' derivatives come from multiplicity-weighted bin sums
(``xy_fss_resample``, ``xy_fss_curves``).  Curves of two sizes cross near
the critical coupling (Sec. III: rho_s L and U_L of different L intersect
at T_c); ``xy_fss_crossings`` locates the crossing of every resample and the
slopes there, which give 1/nu = ln(slope_B / slope_A) / ln(L_B / L_A).

This module marshals arguments only: every step runs in the library's
kernels.  The resample multiplicities are inputs (drawn here on the host
with a seeded generator, so that an independent check can use the same
resamples).
"""

from __future__ import annotations

import numpy as np

from . import xy

N_SUMS = 11
CURVE_ROWS = ("U", "rhoL", "dU", "drhoL")
CROSS_COLS = ("beta", "slopeA", "slopeB", "inv_nu", "nu")


def bootstrap_counts(n_bins: int, n_resamples: int, seed: int, draws: int | None = None) -> np.ndarray:
    """Bin multiplicities of bootstrap resamples: `draws` bins (default
    n_bins) drawn with replacement, int32 [n_resamples][n_bins]."""
    rng = np.random.default_rng(seed)
    d = n_bins if draws is None else int(draws)
    return rng.multinomial(d, np.full(n_bins, 1.0 / n_bins), size=n_resamples).astype(np.int32)


def jackknife_counts(n_bins: int) -> np.ndarray:
    """Leave-one-bin-out multiplicities, int32 [n_bins][n_bins]."""
    return (1 - np.eye(n_bins, dtype=np.int32)).astype(np.int32)


def bin_sums(series, beta0: float, betap, n_bins: int, scratch=None):
    """Per-bin reweighting sums [n_bins][K][11] and {Ebar, min e, max e}."""
    import torch
    E, m2, m4, c, s2 = xy._series_tensors(series)
    bp = torch.as_tensor(betap, dtype=torch.float64, device="cuda").contiguous()
    T, K = E.numel(), bp.numel()
    need = xy.lib().xy_reweight_bins_scratch_bytes(T, K, int(n_bins))
    if need == 0:
        raise xy.XYError(xy.XY_ERR_ARG, "xy_reweight_bins_scratch_bytes")
    if scratch is None or scratch.numel() < need:
        scratch = torch.empty(int(need), dtype=torch.uint8, device="cuda")
    bins = torch.empty((int(n_bins), K, N_SUMS), dtype=torch.float64, device="cuda")
    stats = torch.empty(3, dtype=torch.float64, device="cuda")
    xy._check(xy.lib().xy_reweight_bins(T, E.data_ptr(), m2.data_ptr(), m4.data_ptr(), c.data_ptr(),
                                        s2.data_ptr(), float(beta0), K, bp.data_ptr(), int(n_bins),
                                        bins.data_ptr(), stats.data_ptr(), scratch.data_ptr(),
                                        int(scratch.numel()), torch.cuda.current_stream().cuda_stream),
              "xy_reweight_bins")
    return bins, stats


def resample(bins, counts):
    """Sums of each resample [B][K][11] from bin sums and multiplicities."""
    import torch
    cnt = torch.as_tensor(np.ascontiguousarray(counts, dtype=np.int32), device="cuda").contiguous()
    n_bins, K, _ = bins.shape
    B = cnt.shape[0]
    if cnt.shape[1] != n_bins:
        raise ValueError("counts must be [B][n_bins]")
    out = torch.empty((B, K, N_SUMS), dtype=torch.float64, device="cuda")
    xy._check(xy.lib().xy_fss_resample(n_bins, K, bins.data_ptr(), B, cnt.data_ptr(), out.data_ptr(),
                                       torch.cuda.current_stream().cuda_stream), "xy_fss_resample")
    return out


def curves(sums, betap, L: int):
    """[B][4][K]: U_L, rho_s L and their beta' derivatives per resample."""
    import torch
    bp = torch.as_tensor(betap, dtype=torch.float64, device="cuda").contiguous()
    B, K, _ = sums.shape
    out = torch.empty((B, 4, K), dtype=torch.float64, device="cuda")
    xy._check(xy.lib().xy_fss_curves(B, K, bp.data_ptr(), int(L), sums.data_ptr(), out.data_ptr(),
                                     torch.cuda.current_stream().cuda_stream), "xy_fss_curves")
    return out


def crossings(betap, LA: int, curvesA, LB: int, curvesB, which: str = "U"):
    """[B][5] = {beta*, slope A, slope B, 1/nu, nu} per resample (NaN when
    the two curves do not cross on the grid)."""
    import torch
    bp = torch.as_tensor(betap, dtype=torch.float64, device="cuda").contiguous()
    B, _, K = curvesA.shape
    out = torch.empty((B, 5), dtype=torch.float64, device="cuda")
    w = {"U": 0, "rhoL": 1}[which]
    xy._check(xy.lib().xy_fss_crossings(B, K, bp.data_ptr(), int(LA), curvesA.data_ptr(), int(LB),
                                        curvesB.data_ptr(), w, out.data_ptr(),
                                        torch.cuda.current_stream().cuda_stream), "xy_fss_crossings")
    return out


def analyse(series_by_L: dict, beta0: float, betap, n_bins: int, counts, scratch=None):
    """Crossings of U_L and rho_s L for consecutive sizes, for every
    resample in `counts` ([B][n_bins] multiplicities).  Returns
    {"curves": {L: [B][4][K]}, (LA, LB, which): [B][5], ...} as CUDA
    tensors; summarise with :func:`summary`."""
    Ls = sorted(series_by_L)
    res = {"curves": {}}
    for L in Ls:
        bins, _ = bin_sums(series_by_L[L], beta0, betap, n_bins, scratch)
        res["curves"][L] = curves(resample(bins, counts), betap, L)
    for LA, LB in zip(Ls[:-1], Ls[1:]):
        for which in ("U", "rhoL"):
            res[(LA, LB, which)] = crossings(betap, LA, res["curves"][LA], LB, res["curves"][LB], which)
    return res


def summary(cross, kind: str = "bootstrap") -> dict:
    """Mean and error of each column over the resamples that crossed:
    bootstrap error = standard deviation over resamples (Sec. II: one
    standard deviation); jackknife error = sqrt((n-1)/n sum (x_i - x)^2)."""
    x = cross.detach().cpu().numpy() if hasattr(cross, "detach") else np.asarray(cross)
    ok = np.all(np.isfinite(x), axis=1)
    x = x[ok]
    n = len(x)
    out = {"n": int(n)}
    for j, name in enumerate(CROSS_COLS):
        if n == 0:
            out[name] = (float("nan"), float("nan"))
            continue
        m = float(x[:, j].mean())
        if kind == "jackknife":
            err = float(np.sqrt((n - 1) / n * np.sum((x[:, j] - m) ** 2)))
        else:
            err = float(x[:, j].std(ddof=1)) if n > 1 else float("nan")
        out[name] = (m, err)
    return out
