"""Physics check of the whole path (Sec. III): the library's own sweeps of
L = 8 and 16 near beta_c, reweighted on the device, give U_L and rho_s L
curves that cross near the critical coupling beta_c = 1 / 2.2018 = 0.4542,
with a slope ratio in the range of the 3D XY exponent (1/nu ~ 1.49).
Loose by design: these are small lattices and short runs."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _series(L, sweeps, seed):
    from paper_1211_0780_b300 import xy
    sim = xy.Simulation(L, 1, [0.4542], seed, series_capacity=sweeps)
    sim.set_exec(xy.EXEC_GRAPH)
    sim.sweep(1, 2, 2000)
    sim.read_series()
    sim.sweep(1, 2, sweeps, measure_every=1)
    rec = sim.read_series()
    N = float(L ** 3)
    m2 = (rec["Mx"] ** 2 + rec["My"] ** 2) / N ** 2
    return {"E": rec["E"], "m2": m2.astype(np.float32), "m4": (m2 * m2).astype(np.float32),
            "c": (rec["C"].T / N).astype(np.float32), "s2": (rec["S"].T ** 2 / N).astype(np.float32)}


def test_binder_and_stiffness_cross_near_beta_c():
    from paper_1211_0780_b300 import fss
    series = {8: _series(8, 40000, 31), 16: _series(16, 40000, 32)}
    bp = np.linspace(0.440, 0.470, 301)
    n_bins = 20
    counts = np.concatenate([np.ones((1, n_bins), np.int32), fss.bootstrap_counts(n_bins, 50, seed=1)])
    res = fss.analyse(series, 0.4542, bp, n_bins, counts)
    for which in ("U", "rhoL"):
        x = res[(8, 16, which)].cpu().numpy()
        assert np.isfinite(x[0, 0]), which  # the full series crosses on the window
        assert abs(x[0, 0] - 0.4542) < 0.006, (which, x[0, 0])
        sb = fss.summary(x[1:])
        assert sb["n"] >= 40
        assert abs(sb["beta"][0] - 0.4542) < 0.006
    inv_nu = res[(8, 16, "U")].cpu().numpy()[0, 3]
    assert 1.0 < inv_nu < 2.0, inv_nu
