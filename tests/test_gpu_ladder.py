"""Adaptive ladder on the device: a new ladder installed in a running
context acts exactly like a context created with it, and the adaptation
evens out the measured exchange acceptance of a real parallel-tempering
run."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_set_betas_equals_fresh_context():
    from paper_1211_0780_b300 import xy
    L, R = 8, 4
    a = xy.Simulation(L, R, [0.40, 0.42, 0.44, 0.46], 7, series_capacity=64)
    a.sweep(1, 1, 20, measure_every=0, pt_swap_every=1)
    new = np.array([0.39, 0.43, 0.44, 0.50])
    a.set_betas(0, new)
    b = xy.Simulation(L, R, new, 7, series_capacity=64)
    angles, perm, ctr = a.get_state()
    b.set_packed(a.get_packed())
    b.set_state(None, perm, ctr)
    for s in (a, b):
        s.sweep(1, 2, 6, measure_every=1, pt_swap_every=1)
    assert np.array_equal(a.get_packed(), b.get_packed())
    ra, rb = a.read_series(), b.read_series()
    assert np.array_equal(ra, rb)
    np.testing.assert_array_equal(np.sort(np.unique(ra["beta"])), new)
    assert np.all(new[ra["beta_index"]] == ra["beta"])


def test_adaptation_evens_out_acceptance():
    from paper_1211_0780_b300 import ladder, xy
    L, R = 8, 8
    b0 = np.linspace(0.30, 0.60, R)
    sim = xy.Simulation(L, R, b0, 11)
    sim.sweep(1, 2, 300, pt_swap_every=1)
    hist = ladder.adapt(sim, 0, n_iter=3, sweeps=2000, damping=0.7)
    first, last = hist[0][1], hist[-1][1]
    bl = hist[-1][0]
    assert bl[0] == b0[0] and bl[-1] == b0[-1] and np.all(np.diff(bl) > 0)
    assert np.all((first >= 0) & (first <= 1))
    assert np.ptp(last) < 0.7 * np.ptp(first), (first, last)
