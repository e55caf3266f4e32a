"""Finite-size-scaling path (per-bin reweighting sums, resampling, curves,
crossings) vs the FP64 oracle, which rebuilds every resample as an explicit
series and reweights it exactly."""

import numpy as np
import pytest

import oracle
from oracle import fss as ofss

pytestmark = pytest.mark.gpu

SUM_COLS = {"m2": 3, "m4": 5, "c": 7, "s2": 9}


def _synthetic(L, T, seed):
    from paper_1211_0780_b300.inputs import synthetic_series
    return synthetic_series(L, T, seed)


def test_bin_sums_are_each_bins_reweighting():
    """S[b][k][j] / S[b][k][0] is bin b's reweighted average at beta'_k, and
    the bins add up to the whole series."""
    from paper_1211_0780_b300 import fss, xy
    L, T, n_bins = 16, 12001, 12
    s = _synthetic(L, T, 21)
    beta0 = 0.4542
    bp = np.linspace(0.4500, 0.4590, 40)
    bins, stats = fss.bin_sums(s, beta0, bp, n_bins)
    S = bins.cpu().numpy()
    Ebar = float(stats[0])
    edges = ofss.bin_edges(T, n_bins)
    for b in range(n_bins):
        sub = {k: (v[..., edges[b]:edges[b + 1]] if isinstance(v, np.ndarray) else v) for k, v in s.items()}
        ref = ofss.curves_at(sub, beta0, bp, L)
        for name, j in SUM_COLS.items():
            np.testing.assert_allclose(S[b, :, j] / S[b, :, 0], ref[name], rtol=1e-10, err_msg=f"bin {b} {name}")
        np.testing.assert_allclose(Ebar + S[b, :, 1] / S[b, :, 0], ref["E"], rtol=1e-12)
    tot = S.sum(axis=0)
    ref = ofss.curves_at(s, beta0, bp, L)
    np.testing.assert_allclose(tot[:, 3] / tot[:, 0], ref["m2"], rtol=1e-10)
    f = xy.reweight_forward(s, beta0, bp, L)
    np.testing.assert_allclose(tot[:, 5] / tot[:, 0], f["m4"].cpu().numpy(), rtol=1e-10)


@pytest.mark.parametrize("n_bins,T", [(10, 5000), (7, 4003)])
def test_resampled_curves_match_oracle(n_bins, T):
    from paper_1211_0780_b300 import fss
    L = 24
    s = _synthetic(L, T, 5 + n_bins)
    beta0 = 0.4542
    bp = np.linspace(0.4510, 0.4575, 33)
    counts = np.concatenate([np.ones((1, n_bins), np.int32), fss.bootstrap_counts(n_bins, 5, seed=9),
                             fss.jackknife_counts(n_bins)[:2]])
    bins, _ = fss.bin_sums(s, beta0, bp, n_bins)
    cur = fss.curves(fss.resample(bins, counts), bp, L).cpu().numpy()
    for r, row in enumerate(counts):
        ref = ofss.curves_at(ofss.resampled_series(s, n_bins, row), beta0, bp, L)
        for i, name in enumerate(fss.CURVE_ROWS):
            scale = np.max(np.abs(ref[name]))
            np.testing.assert_allclose(cur[r, i], ref[name], rtol=1e-9, atol=1e-9 * scale,
                                       err_msg=f"resample {r} {name}")


def _simulated_series(L, sweeps, seed):
    """A series from the library's own sweeps at beta0 (1 Metropolis + 2
    over-relaxation passes, measured every sweep)."""
    from paper_1211_0780_b300 import xy
    sim = xy.Simulation(L, 1, [0.4542], seed, series_capacity=sweeps)
    sim.set_exec(xy.EXEC_GRAPH)
    sim.sweep(1, 2, 400)
    sim.read_series()
    sim.sweep(1, 2, sweeps, measure_every=1)
    rec = sim.read_series()
    N = float(L ** 3)
    m2 = (rec["Mx"] ** 2 + rec["My"] ** 2) / N ** 2
    return {"E": rec["E"].astype(np.float64), "m2": m2.astype(np.float32), "m4": (m2 * m2).astype(np.float32),
            "c": (rec["C"].T / N).astype(np.float32), "s2": (rec["S"].T ** 2 / N).astype(np.float32)}


def test_crossings_of_simulated_sizes_match_oracle():
    """U_L and rho_s L of L = 8 and 16 (the library's own sweeps near
    beta_c): the crossing, the slopes there and 1/nu of every resample agree
    with the oracle's exact root of the reweighted curves."""
    from paper_1211_0780_b300 import fss
    beta0, n_bins = 0.4542, 10
    series = {8: _simulated_series(8, 4000, 101), 16: _simulated_series(16, 4000, 202)}
    bp = np.linspace(0.430, 0.480, 401)
    counts = np.concatenate([np.ones((1, n_bins), np.int32), fss.bootstrap_counts(n_bins, 3, seed=4)])
    res = fss.analyse(series, beta0, bp, n_bins, counts)
    crossed = 0
    for which in ("U", "rhoL"):
        got = res[(8, 16, which)].cpu().numpy()
        for r, row in enumerate(counts):
            sA = ofss.resampled_series(series[8], n_bins, row)
            sB = ofss.resampled_series(series[16], n_bins, row)
            ref = ofss.crossing(sA, 8, sB, 16, beta0, bp, which)
            if np.isnan(ref[0]):
                assert np.isnan(got[r, 0]), (which, r)
                continue
            crossed += 1
            assert got[r, 0] == pytest.approx(ref[0], abs=1e-9), (which, r)
            assert got[r, 1] == pytest.approx(ref[1], rel=1e-6)
            assert got[r, 2] == pytest.approx(ref[2], rel=1e-6)
            assert got[r, 3] == pytest.approx(ref[3], rel=1e-5, abs=1e-6)
    assert crossed >= 4  # the curves do cross near beta_c for most resamples


def test_summary_errors():
    from paper_1211_0780_b300 import fss
    x = np.array([[0.45, 1.0, 2.0, 1.5, 1 / 1.5], [0.46, 1.1, 2.1, 1.4, 1 / 1.4],
                  [np.nan] * 5, [0.44, 0.9, 1.9, 1.6, 1 / 1.6]])
    sb = fss.summary(x)
    assert sb["n"] == 3
    assert sb["beta"][0] == pytest.approx(0.45) and sb["beta"][1] == pytest.approx(0.01)
    sj = fss.summary(x, kind="jackknife")
    assert sj["inv_nu"][1] == pytest.approx(np.sqrt(2 / 3 * 0.02))
