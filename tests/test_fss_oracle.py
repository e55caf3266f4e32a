"""Pins of the finite-size-scaling oracle (CPU): crossings and 1/nu of
curves that follow the scaling form of Sec. III exactly, the resampled
series, and the jackknife and bootstrap errors of a plain mean."""

import numpy as np
import pytest

from oracle import fss as ofss
import oracle


def _scaling_pair(F, dF, bc, nu, LA, LB):
    def mk(L):
        s = L ** (1.0 / nu)
        return (lambda b: F((b - bc) * s)), (lambda b: dF((b - bc) * s) * s)
    return mk(LA) + mk(LB)


@pytest.mark.parametrize("LA,LB", [(16, 32), (64, 80), (128, 160)])
def test_crossing_of_exact_scaling_curves(LA, LB):
    """Q_L(beta) = F((beta - beta_c) L^{1/nu}) for every L: all sizes cross
    at beta_c and the slope ratio gives nu exactly (Sec. III, Eq. 7)."""
    bc, nu = 0.4542, 0.6717
    for F, dF in ((lambda x: np.tanh(3 * x) + 0.4, lambda x: 3 / np.cosh(3 * x) ** 2),
                  (lambda x: 1 / (1 + np.exp(-x)), lambda x: np.exp(-x) / (1 + np.exp(-x)) ** 2)):
        fA, dA, fB, dB = _scaling_pair(F, dF, bc, nu, LA, LB)
        # a window a few scaling widths wide (the curves saturate far out)
        w = 3.0 * LA ** (-1.0 / nu)
        grid = np.linspace(bc - w, bc + 1.1 * w, 61)
        b, sA, sB, inv_nu, got_nu = ofss.crossing_of(fA, dA, fB, dB, grid, LA, LB)
        assert b == pytest.approx(bc, abs=1e-13)
        assert got_nu == pytest.approx(nu, rel=1e-12)
        assert sB / sA == pytest.approx((LB / LA) ** (1 / nu), rel=1e-12)


def test_no_crossing_gives_nan():
    grid = np.linspace(0.44, 0.47, 11)
    r = ofss.crossing_of(lambda b: b, lambda b: 1.0, lambda b: b + 1, lambda b: 1.0, grid, 8, 16)
    assert all(np.isnan(v) for v in r)


def _series(T, seed):
    from paper_1211_0780_b300.inputs import synthetic_series
    s = synthetic_series(16, T, seed)
    return s


def test_resampled_series_repeats_whole_bins():
    s = _series(1000, 3)
    same = ofss.resampled_series(s, 10, np.ones(10, int))
    assert np.array_equal(same["E"], s["E"]) and np.array_equal(same["c"], s["c"].astype(np.float64))
    cnt = np.zeros(10, int)
    cnt[3], cnt[7] = 2, 1
    r = ofss.resampled_series(s, 10, cnt)
    assert np.array_equal(r["E"], np.concatenate([s["E"][300:400], s["E"][300:400], s["E"][700:800]]))


def test_jackknife_error_of_a_plain_mean_is_the_standard_error():
    """At beta' = beta0 reweighting returns plain means; the leave-one-bin-
    out estimates of a mean over equal bins have jackknife error exactly
    s / sqrt(n) of the bin means."""
    from paper_1211_0780_b300.fss import jackknife_counts
    s = _series(2400, 5)
    n, beta0 = 12, 0.4542
    vals = []
    for row in jackknife_counts(n):
        r = ofss.resampled_series(s, n, row)
        vals.append(ofss.curves_at(r, beta0, [beta0], 16)["m2"][0])
    vals = np.array(vals)
    jk = np.sqrt((n - 1) / n * np.sum((vals - vals.mean()) ** 2))
    bin_means = np.asarray(s["m2"], np.float64).reshape(n, -1).mean(axis=1)
    assert jk == pytest.approx(bin_means.std(ddof=1) / np.sqrt(n), rel=1e-10)


def test_bootstrap_error_of_a_plain_mean():
    """Bootstrap over bins (n draws with replacement): the spread of the
    resampled mean is sqrt((n - 1) / n) s / sqrt(n) (statistically, 4000
    resamples: within 5%)."""
    from paper_1211_0780_b300.fss import bootstrap_counts
    rng = np.random.default_rng(11)
    n = 40
    x = rng.gamma(3.0, 1.0, size=n)
    cnt = bootstrap_counts(n, 4000, seed=2)
    assert np.all(cnt.sum(axis=1) == n)
    means = cnt @ x / n
    want = np.sqrt((n - 1) / n) * x.std(ddof=1) / np.sqrt(n)
    assert means.std() == pytest.approx(want, rel=0.05)
