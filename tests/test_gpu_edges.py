"""Edge cases of the analysis kernels: one bin, two couplings, one
resample, unequal record counts, the largest ladder, and argument checks."""

import numpy as np
import pytest

from oracle import fss as ofss
from oracle import multihist as omh

pytestmark = pytest.mark.gpu


def _synthetic(L, T, seed):
    from paper_1211_0780_b300.inputs import synthetic_series
    return synthetic_series(L, T, seed)


def test_single_bin_two_couplings_one_resample():
    from paper_1211_0780_b300 import fss
    s = _synthetic(16, 3001, 4)
    bp = np.array([0.4530, 0.4555])
    bins, _ = fss.bin_sums(s, 0.4542, bp, 1)
    cur = fss.curves(fss.resample(bins, np.ones((1, 1), np.int32)), bp, 16).cpu().numpy()
    ref = ofss.curves_at(s, 0.4542, bp, 16)
    np.testing.assert_allclose(cur[0, 0], ref["U"], rtol=1e-9)
    np.testing.assert_allclose(cur[0, 1], ref["rhoL"], rtol=1e-9)


def test_bins_as_many_as_samples_and_zero_multiplicities():
    from paper_1211_0780_b300 import fss
    s = _synthetic(8, 64, 5)
    bp = np.linspace(0.445, 0.462, 9)
    bins, _ = fss.bin_sums(s, 0.4542, bp, 64)  # one sample per bin
    counts = np.zeros((2, 64), np.int32)
    counts[0, :] = 1
    counts[1, ::2] = 2  # even samples twice, odd ones dropped
    cur = fss.curves(fss.resample(bins, counts), bp, 8).cpu().numpy()
    for r in range(2):
        ref = ofss.curves_at(ofss.resampled_series(s, 64, counts[r]), 0.4542, bp, 8)
        np.testing.assert_allclose(cur[r, 0], ref["U"], rtol=1e-9)


def test_reweighting_argument_checks():
    from paper_1211_0780_b300 import fss, xy
    s = _synthetic(8, 100, 6)
    with pytest.raises(xy.XYError):
        fss.bin_sums(s, 0.45, [0.45, 0.46], 101)  # more bins than samples
    with pytest.raises(xy.XYError):
        fss.bin_sums(s, 0.45, [0.45, 0.46], 0)


def test_multihist_unequal_counts_and_largest_ladder():
    from paper_1211_0780_b300 import multihist as mh
    rng = np.random.default_rng(8)
    R = 64
    betas = np.linspace(0.40, 0.50, R)
    n = rng.integers(200, 600, R)
    s = 60.0
    parts = []
    for b, k in zip(betas, n):
        E = -4000.0 - b * s * s + s * rng.standard_normal(k)
        m2 = np.clip(0.05 + 0.001 * rng.standard_normal(k), 0, 1)
        parts.append({"E": E, "m2": m2.astype(np.float32), "m4": (m2 * m2).astype(np.float32),
                      "c": np.full((3, k), 0.4, np.float32), "s2": np.full((3, k), 0.1, np.float32)})
    pooled, counts = mh.pool(parts)
    f, it = mh.solve(pooled, betas, counts, tol=1e-11)
    fo, _ = omh.solve(pooled["E"], betas, counts, tol=1e-13)
    np.testing.assert_allclose(f, fo, atol=1e-8)
    with pytest.raises(Exception):
        mh.solve(pooled, np.linspace(0.40, 0.50, 65), np.append(counts, 1))  # 65 couplings


def test_ladder_two_replicas_and_bad_betas():
    from paper_1211_0780_b300 import ladder, xy
    np.testing.assert_array_equal(ladder.update([0.4, 0.5], [0.3]), [0.4, 0.5])
    sim = xy.Simulation(8, 3, [0.40, 0.42, 0.44], 3)
    with pytest.raises(xy.XYError):
        sim.set_betas(0, [0.40, 0.39, 0.44])
    sim.set_betas(0, [0.41, 0.42, 0.43])
    np.testing.assert_array_equal(sim.ladder(0), [0.41, 0.42, 0.43])


def test_autotune_cache_reuses_tiles(tmp_path):
    """A second context with the same lattices, passes and mode takes its
    tiles from the JSON cache (xy_set_tile) and gets the first one's."""
    from paper_1211_0780_b300 import xy
    path = str(tmp_path / "tiles.json")
    a = xy.Simulation(24, 2, [0.44, 0.45], 7)
    t1 = a.autotune(1, 1, cache=path)
    b = xy.Simulation(24, 2, [0.44, 0.45], 8)
    t2 = b.autotune(1, 1, cache=path)
    assert t1 == t2 == [b.get_tile(0)]
    assert len(xy.load_tile_cache(path)) == 1
    b.set_exec(xy.EXEC_GRAPH)
    b.autotune(1, 1, cache=path)  # another mode: another entry
    assert len(xy.load_tile_cache(path)) == 2


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_autotune_leaves_the_state(mode):
    """Autotuning runs trial sweeps (whole sweeps with an exchange at every
    sweep's end in each execution mode: plain launches, the CUDA graph,
    persistent launches) but restores the spins, the ladder's permutation
    and couplings, and the counters and accept counts: the context then
    sweeps exactly as a fresh one set to the tiles autotune chose."""
    from paper_1211_0780_b300 import xy
    betas = [0.42, 0.44, 0.46, 0.48]
    a = xy.Simulation([16, 24], [4, 2], betas + [0.44, 0.45], 11, series_capacity=16)
    a.set_exec(mode)
    a.sweep(1, 2, 3, pt_swap_every=1)
    before = (a.get_packed(), a.get_state()[1], a.get_state()[2], a.accepts())
    tiles = a.autotune(1, 2)
    after = (a.get_packed(), a.get_state()[1], a.get_state()[2], a.accepts())
    assert np.array_equal(before[0], after[0])
    assert np.array_equal(before[1], after[1])
    assert np.array_equal(before[2], after[2])
    assert np.array_equal(before[3][0], after[3][0]) and np.array_equal(before[3][1], after[3][1])
    b = xy.Simulation([16, 24], [4, 2], betas + [0.44, 0.45], 11, series_capacity=16)
    b.set_exec(mode)
    b.sweep(1, 2, 3, pt_swap_every=1)
    for i, (ty, tz, kind) in enumerate(tiles):
        b.set_tile(i, ty, tz, kind)
    for s in (a, b):
        s.sweep(1, 2, 4, measure_every=2, pt_swap_every=1)
    assert np.array_equal(a.get_packed(), b.get_packed())
    assert np.array_equal(a.get_state()[1], b.get_state()[1])
    assert a.read_series().tobytes() == b.read_series().tobytes()


def test_readme_usage_runs():
    """The usage example of the README at a small size: ladder run, series
    split by coupling, differentiable reweighting, checkpoint and resume."""
    import torch
    from paper_1211_0780_b300 import multihist, xy
    L, R = 16, 4
    betas = np.linspace(0.450, 0.458, R)
    sim = xy.Simulation(L, R, betas, seed=0x5EED2012)
    sim.set_exec(xy.EXEC_GRAPH)
    sim.autotune(1, 3)
    sim.sweep(1, 3, 20, measure_every=1, pt_swap_every=1)
    rec = sim.read_series()
    assert len(rec) == 20 * R
    series, b = multihist.series_from_records(rec, L, R)
    bp = torch.linspace(0.4530, 0.4555, 64, dtype=torch.float64, device="cuda", requires_grad=True)
    U, rhoL = xy.reweight(series[2], b[2], bp, L)
    U.sum().backward()
    assert torch.isfinite(bp.grad).all() and torch.isfinite(rhoL).all()
    packed = sim.get_packed()
    _, perm, counters = sim.get_state()
    resumed = xy.Simulation(L, R, betas, seed=0x5EED2012)
    resumed.set_packed(packed)
    resumed.set_state(None, perm, counters)
    sim.sweep(1, 3, 3, measure_every=1, pt_swap_every=1)
    resumed.sweep(1, 3, 3, measure_every=1, pt_swap_every=1)
    assert np.array_equal(sim.get_packed(), resumed.get_packed())
    assert sim.read_series().tobytes() == resumed.read_series().tobytes()


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_empty_and_rejected_sweeps_change_nothing(mode):
    """Zero sweeps is a no-op; zero passes per sweep and a series buffer
    too small for the requested records are rejected before any work (the
    state, counters and series stay as they were and the context stays
    usable); a one-replica ladder with exchanges requested has no pair to
    exchange and keeps its permutation."""
    from paper_1211_0780_b300 import xy
    sim = xy.Simulation([8, 16], [1, 3], [0.45, 0.44, 0.45, 0.46], seed=11, series_capacity=4)
    sim.set_exec(mode)
    sim.sweep(1, 2, 2, measure_every=1, pt_swap_every=1)
    before = (sim.get_packed().copy(), sim.counters().copy(), sim.series_count())
    _, perm0, _ = sim.get_state()

    def unchanged():
        return (np.array_equal(sim.get_packed(), before[0]) and np.array_equal(sim.counters(), before[1])
                and sim.series_count() == before[2])

    sim.sweep(1, 2, 0, measure_every=1, pt_swap_every=1)
    assert unchanged()
    with pytest.raises(xy.XYError) as e:
        sim.sweep(0, 0, 3)
    assert e.value.status == xy.XY_ERR_ARG and unchanged()
    with pytest.raises(xy.XYError) as e:
        sim.sweep(1, 2, 3, measure_every=1)  # 2 records buffered + 3 more > capacity 4
    assert e.value.status == xy.XY_ERR_NOMEM and unchanged()
    assert sim.device_status() == 0
    sim.sweep(1, 2, 2, measure_every=1, pt_swap_every=1)  # still usable: fills the buffer
    rec = sim.read_series()
    assert len(rec) == 4 * 4 and np.all(np.isfinite(rec["E"]))
    _, perm1, _ = sim.get_state()
    assert perm1[0] == perm0[0] == 0  # the 8^3 lattice's one-replica ladder
    assert sorted(perm1[1:]) == [0, 1, 2]
