"""Parity at the full sizes of the benchmark workloads, in the launch
configurations bench.py times: the 160^3 lattice on the march tile 8 x 8 in
a CUDA graph, the 64^3 x 32 parallel-tempering batch with its autotuned
tile, the ragged batch in one persistent launch, and reweighting of 10^6
samples to 4096 couplings.  The oracle runs whole half-sweeps of these
lattices (FP64 C), or the sampled couplings for reweighting; tolerances as
in test_gpu_parity (the oracle runs on the exact angles of the stored
vectors; Metropolis: 1e-5 rad outside accept margins < 1e-6; over-relaxation:
the conditioning bound at every site and 99.9% of the sites within 1e-5 rad;
sums: 2e-6 per bond term)."""

import numpy as np
import pytest

import oracle
from helpers import circ_dist, stored_angles64

pytestmark = pytest.mark.gpu

SEED = 0x5EED2012
TOL_RAD, MARGIN = 1e-5, 1e-6
OR_A, OR_B = 8.4e-6, 1e-6  # the conditioning bound of test_gpu_parity
OR_A_ANG, OR_B_ANG = 7.6e-6, 2.8e-6  # the angle tile kind's (test_gpu_angle)
BOND_TOL = 2e-6


def field_norm(theta):
    c, s = np.cos(theta), np.sin(theta)
    hx = sum(np.roll(c, sh, ax) for ax in range(3) for sh in (1, -1))
    hy = sum(np.roll(s, sh, ax) for ax in range(3) for sh in (1, -1))
    return np.hypot(hx, hy)


def colour_mask(L, colour):
    z, y, x = np.meshgrid(*(np.arange(L),) * 3, indexing="ij")
    return ((x + y + z) % 2) == colour


def check_or_half(before, after, colour, angles=False):
    """before, after: exact angles of the stored spins (stored_angles64);
    angles: the lattice is on the angle tile kind."""
    ref = before.copy()
    h = field_norm(ref)
    oracle.overrelax_half(ref, colour)
    d = circ_dist(after, ref)
    m = colour_mask(before.shape[0], colour)
    a, b = (OR_A_ANG, OR_B_ANG) if angles else (OR_A, OR_B)
    assert np.all(d[m] <= a / h[m] + b), float(np.max(d[m] * h[m]))
    assert np.quantile(d[m], 0.999) < TOL_RAD
    assert np.all(d[~m] == 0)


def check_met_half(before, after, beta, slot, mpass, colour):
    ref = before.copy()
    _, margin = oracle.metropolis_half(ref, beta, SEED, slot, mpass, colour, want_margin=True)
    close = margin < MARGIN
    d = circ_dist(after, ref)
    assert np.max(d[~close]) < TOL_RAD
    return int(close.sum())


@pytest.mark.parametrize("kind", [0, 3])
def test_L160_tile_graph(kind):
    """160^3, tile 8 x 8 (march, and direct: the bench's launch shape),
    CUDA graph, 1 + 5 passes: the graph's sweep equals the same half-sweeps
    issued one by one, and each kind of half-sweep and the lattice sums
    agree with the oracle on the full lattice."""
    from paper_1211_0780_b300 import xy
    L, beta = 160, 0.4542
    a = xy.Simulation(L, 1, [beta], SEED, series_capacity=16)
    a.set_tile(0, 8, 8, kind)
    a.set_exec(xy.EXEC_GRAPH)
    a.sweep(1, 5, 2, measure_every=1)
    b = xy.Simulation(L, 1, [beta], SEED, series_capacity=16)
    b.set_tile(0, 8, 8, kind)
    _, perm, ctr = a.get_state()
    b.set_packed(a.get_packed())
    b.set_state(None, perm, ctr)
    a.read_series()
    a.sweep(1, 5, 1, measure_every=1)
    mp = int(ctr[0])
    for c in (0, 1):
        b.metropolis_half(c, mp)
    for _ in range(5):
        for c in (0, 1):
            b.overrelax_half(c)
    assert np.array_equal(a.get_packed(), b.get_packed())
    assert a.read_series()["E"][0] == pytest.approx(b.measure()["E"][0], rel=1e-9)

    pk = b.get_packed()
    th = stored_angles64(b, pk)[0]
    b.overrelax_half(0)
    check_or_half(th, stored_angles64(b)[0], 0)
    b.set_packed(pk)
    b.metropolis_half(1, 7)
    excluded = check_met_half(th, stored_angles64(b)[0], beta, 0, 7, 1)
    assert excluded <= 1e-4 * L ** 3 / 2
    b.set_packed(pk)
    s = oracle.measure(th)
    assert abs(b.measure()["E"][0] - s.E) < BOND_TOL * 3 * L ** 3


def test_pt_batch_64cubed_32_replicas():
    """64^3 x 32 on the autotuned tile in a CUDA graph: half-sweeps of every
    replica at its own coupling and the exchange decisions of Eq. 3 agree
    with the oracle."""
    from paper_1211_0780_b300 import xy
    L, R = 64, 32
    betas = np.linspace(0.450, 0.458, R)
    s = xy.Simulation(L, R, betas, SEED, series_capacity=16)
    s.set_exec(xy.EXEC_GRAPH)
    s.autotune(1, 3)
    s.sweep(1, 3, 2, measure_every=1, pt_swap_every=1)
    _, perm, ctr = s.get_state()
    beta_of_slot = np.empty(R)
    beta_of_slot[perm] = betas
    pk = s.get_packed()
    angles = stored_angles64(s, pk)
    s.overrelax_half(1)
    after = stored_angles64(s)
    for slot in range(R):
        check_or_half(angles[slot], after[slot], 1)
    s.set_packed(pk)
    s.metropolis_half(0, 5)
    after = stored_angles64(s)
    excluded = sum(check_met_half(angles[slot], after[slot], beta_of_slot[slot], slot, 5, 0) for slot in range(R))
    assert excluded <= 1e-4 * R * L ** 3 / 2
    # one exchange event on the measured energies
    s.set_packed(pk)
    E = np.array([oracle.measure(a).E for a in angles])
    gE = s.measure()["E"]
    assert np.max(np.abs(gE - E)) < BOND_TOL * 3 * L ** 3
    parity = int(ctr[2]) & 1
    p_ref = perm.astype(np.int32).copy()
    n_ref, _ = oracle.pt_swap(betas, gE, p_ref, SEED, 0, int(ctr[2]), parity)
    tie = any(abs(oracle.pt_uniform(SEED, 0, int(ctr[2]), k)
                  - min(1.0, np.exp((betas[k] - betas[k + 1]) * (gE[perm[k]] - gE[perm[k + 1]])))) < MARGIN
              for k in range(parity, R - 1, 2))
    n = s.pt_swap(parity)
    if not tie:
        assert n == n_ref and np.array_equal(s.get_state()[1], p_ref)


def test_ragged_batch_persistent_launch():
    """L in {16, 24, 32, 48, 64, 96, 128} x 16 replicas: one persistent
    launch per call (autotuned block tiles) gives bit-identical states and
    records to the graph path, and over-relaxation half-sweeps of sampled
    replicas agree with the oracle."""
    from paper_1211_0780_b300 import xy
    Ls = [16, 24, 32, 48, 64, 96, 128]
    R = 16
    betas = np.concatenate([np.linspace(0.452, 0.456, R)] * len(Ls))
    runs = []
    for mode in (xy.EXEC_PERSISTENT, xy.EXEC_GRAPH):
        s = xy.Simulation(Ls, [R] * len(Ls), betas, SEED, series_capacity=8)
        s.set_exec(mode)
        if mode == xy.EXEC_PERSISTENT:
            tiles = s.autotune(1, 3)
        else:
            for i, (ty, tz, kind) in enumerate(tiles):
                s.set_tile(i, ty, tz, kind)
        s.sweep(1, 3, 2, measure_every=1, pt_swap_every=1)
        runs.append((s.get_packed(), s.read_series(), s))
    assert np.array_equal(runs[0][0], runs[1][0])
    assert np.array_equal(runs[0][1], runs[1][1])
    s = runs[1][2]
    angles = stored_angles64(s)
    s.overrelax_half(0)
    after = stored_angles64(s)
    slot0 = np.cumsum([0] + [R] * len(Ls))[:-1]
    for i in (0, 3, 6):  # L = 16, 48, 128, first replica
        check_or_half(angles[slot0[i]], after[slot0[i]], 0, angles=s.get_tile(i)[2] == 4)


def test_reweighting_full_size():
    """T = 10^6 samples to K = 4096 couplings: sampled couplings (every
    256th and both ends) against the oracle's FP64 reweighting."""
    from paper_1211_0780_b300 import xy
    from paper_1211_0780_b300.inputs import synthetic_series
    L, T, K = 160, 10 ** 6, 4096
    s = synthetic_series(L, T, 260)
    bp = np.linspace(0.4530, 0.4555, K)
    f = xy.reweight_forward(s, 0.4542, bp, L)
    _, dobs = xy.reweight_backward(bp, L, f)
    idx = np.unique(np.concatenate([np.arange(0, K, 256), [K - 1]]))
    ref = oracle.reweight_observables(s["E"], s["m2"], s["m4"], s["c"].T, s["s2"].T, 0.4542, bp[idx], L)
    for key in ("E", "m2", "U", "rhoL", "logZ"):
        np.testing.assert_allclose(f[key].cpu().numpy()[idx], ref[key], rtol=1e-10, err_msg=key)
    for row, key in ((0, "dU"), (1, "drhoL")):
        np.testing.assert_allclose(dobs[row].cpu().numpy()[idx], ref[key], rtol=1e-8,
                                   atol=1e-8 * np.max(np.abs(ref[key])))


def test_fss_binned_full_size_sampled():
    """The FSS stage's configuration (10^6 samples in 200 bins, 4096
    couplings, bootstrap resamples): one bin's averages and two resamples'
    curves at sampled couplings against the oracle."""
    from paper_1211_0780_b300 import fss
    from oracle import fss as ofss
    from paper_1211_0780_b300.inputs import synthetic_series
    L, T, K, n_bins = 128, 10 ** 6, 4096, 200
    s = synthetic_series(L, T, 228)
    bp = np.linspace(0.4530, 0.4555, K)
    idx = np.arange(0, K, 512)
    bins, stats = fss.bin_sums(s, 0.4542, bp, n_bins)
    S = bins.cpu().numpy()
    edges = ofss.bin_edges(T, n_bins)
    b = 137
    sub = {k: (v[..., edges[b]:edges[b + 1]] if isinstance(v, np.ndarray) else v) for k, v in s.items()}
    ref = ofss.curves_at(sub, 0.4542, bp[idx], L)
    np.testing.assert_allclose(S[b, idx, 3] / S[b, idx, 0], ref["m2"], rtol=1e-10)
    counts = fss.bootstrap_counts(n_bins, 2, seed=3)
    cur = fss.curves(fss.resample(bins, counts), bp, L).cpu().numpy()
    for r in range(2):
        ref = ofss.curves_at(ofss.resampled_series(s, n_bins, counts[r]), 0.4542, bp[idx], L)
        np.testing.assert_allclose(cur[r, 0, idx], ref["U"], rtol=1e-9)
        np.testing.assert_allclose(cur[r, 1, idx], ref["rhoL"], rtol=1e-9)


def test_multihist_full_size_is_a_fixed_point_of_the_oracle_equations():
    """The multi-histogram stage's configuration (32^3 x 32 ladder, 3000
    measured sweeps): the device's free energies satisfy the oracle's
    Ferrenberg-Swendsen equations (one textbook update moves them by < 1e-8),
    and averages at sampled couplings agree with the oracle's."""
    from paper_1211_0780_b300 import multihist as mh, xy
    from oracle import multihist as omh
    from scipy.special import logsumexp
    L, R = 32, 32
    betas = np.linspace(0.440, 0.468, R)
    sim = xy.Simulation(L, R, betas, SEED, series_capacity=3000)
    sim.set_exec(xy.EXEC_GRAPH)
    sim.sweep(1, 3, 500, pt_swap_every=1)
    sim.read_series()
    sim.sweep(1, 3, 3000, measure_every=1, pt_swap_every=1)
    parts, b = mh.series_from_records(sim.read_series(), L, R)
    pooled, counts = mh.pool(parts)
    f, it = mh.solve(pooled, b, counts, tol=1e-11)
    lD = omh.log_denominator(pooled["E"], b, counts, f)
    fn = -logsumexp(-b[None, :] * pooled["E"][:, None] - lD[:, None], axis=0)
    fn -= fn[0]
    assert np.max(np.abs(fn - f)) < 1e-8
    bp = np.linspace(0.440, 0.468, 9)
    g = mh.forward(pooled, b, counts, f, bp, L)
    mE, _, _ = omh.averages(pooled["E"], pooled["E"][:, None], b, counts, f, bp)
    np.testing.assert_allclose(g["E"].cpu().numpy(), mE, rtol=1e-10)


def test_large_lattice_properties():
    """L = 512 (134M sites, beyond every benchmark size): an over-relaxation
    half-sweep conserves the energy, applying it twice returns the state
    (the reflection is an involution with the field frozen), and the
    Metropolis half-sweep touches only its colour.  Properties that hold at
    any size; index arithmetic past 2^26 sites per colour."""
    from paper_1211_0780_b300 import xy
    L = 512
    s = xy.Simulation(L, 1, [0.4542], SEED, series_capacity=4)
    s.sweep(1, 1, 2)
    E0 = s.measure()["E"][0]
    pk0 = s.get_packed()
    s.overrelax_half(0)
    E1 = s.measure()["E"][0]
    assert abs(E1 - E0) < 1e-6 * abs(E0)
    s.overrelax_half(0)
    pk2 = s.get_packed()
    half = L ** 3 // 2
    # colour 1 untouched bit for bit, colour 0 back to within FP32 rounding
    assert np.array_equal(pk2[2 * half:], pk0[2 * half:])
    dc = np.abs(pk2[:half] - pk0[:half])
    ds = np.abs(pk2[half:2 * half] - pk0[half:2 * half])
    assert np.mean(np.maximum(dc, ds) > 1e-5) < 1e-3
    s.set_packed(pk0)
    s.metropolis_half(1, 3)
    pk3 = s.get_packed()
    assert np.array_equal(pk3[:2 * half], pk0[:2 * half])
    assert not np.array_equal(pk3[2 * half:], pk0[2 * half:])
