"""Accuracy of the FP32 fast-math path against FP64, stated as measured
numbers with asserted bounds.

1. The fast intrinsics of the Metropolis update (Sec. II), evaluated by the
   same device functions the sweep kernels inline (xy_debug_fast_math):
   the proposal vector of every one of the 2^24 proposal words, and the
   acceptance threshold exp(x) 2^24 over the exponents x = -beta dE reached.
   Also the angle-storage tile's atan2 over the plane.
2. The error of each measured observable against the FP64 oracle on the
   same stored states: the lattice sums E, M, C_mu, S_mu of every record
   (Eqs. 4-6), U_L and rho_s of the series (Eqs. 5-6), and the reweighted
   U_L, rho_s L and their beta' derivatives.

Each test prints its table (pytest -s shows it).
"""

import numpy as np
import pytest

import oracle
from helpers import stored_angles64

pytestmark = pytest.mark.gpu

SEED = 0x5EED2012


def test_proposal_vectors_of_every_word():
    """All 2^24 proposal values: theta' = (w >> 8) 2 pi / 2^24 (an FP32
    product) turned into (cos, sin) by the fast sincos at theta' - pi.
    Against cos and sin of the exact 2 pi k / 2^24: the FP32 product
    k (2 pi / 2^24) rounds theta' by <= half an ulp (<= 2.4e-7 rad below
    2 pi; the constant itself is fl(2 pi) / 2^24, off by 2.8e-8 relative),
    theta' - pi is formed with fl(pi), off by 8.7e-8, and the fast sincos
    adds its documented absolute error on [-pi, pi], 2^-21.41 = 3.6e-7, per
    component: bound 7e-7 on the direction and on each component.  The
    vector's length error, which the over-relaxation tolerance takes as
    <= 5e-7, is asserted too."""
    from paper_1211_0780_b300 import xy
    k = np.arange(1 << 24, dtype=np.uint32)
    v = xy.fast_math("proposal", k << np.uint32(8)).astype(np.float64)
    th = 2 * np.pi * k.astype(np.float64) / 2.0 ** 24
    ec = np.abs(v[:, 0] - np.cos(th))
    es = np.abs(v[:, 1] - np.sin(th))
    da = np.abs(np.mod(np.arctan2(v[:, 1], v[:, 0]) - th + np.pi, 2 * np.pi) - np.pi)
    dl = np.abs(np.hypot(v[:, 0], v[:, 1]) - 1.0)
    print(f"\nproposal vectors, 2^24 words: max |dcos| {ec.max():.3e}, max |dsin| {es.max():.3e}, "
          f"max direction error {da.max():.3e} rad (rms {np.sqrt(np.mean(da ** 2)):.3e}), "
          f"max ||v| - 1| {dl.max():.3e}")
    assert da.max() <= 7e-7
    assert max(ec.max(), es.max()) <= 7e-7
    assert dl.max() <= 5e-7


def test_acceptance_threshold_exponential():
    """exp(x) 2^24 with the fast exponential, against FP64 exp(x) 2^24.
    Bound: the documented ulp error of the fast exponential, 2 + |1.173 x|
    ulp, i.e. a relative error <= (2 + 1.2 |x|) 2^-23.  Reported over the
    exponents the update reaches at the paper's couplings (|x| = beta |dE|
    <= 12 beta: |x| <= 6 for beta <= 0.5) and over [-30, 6]."""
    from paper_1211_0780_b300 import xy
    rng = np.random.default_rng(7)
    x = np.concatenate([np.linspace(-30.0, 6.0, 1 << 22), rng.uniform(-6.0, 6.0, 1 << 22),
                        np.linspace(-1e-3, 1e-3, 4097)]).astype(np.float32)
    t = xy.fast_math("accept", x).astype(np.float64)
    ref = np.exp(x.astype(np.float64)) * 2.0 ** 24
    rel = np.abs(t - ref) / ref
    inrange = np.abs(x) <= 6.0
    print(f"\nacceptance threshold exp(x) 2^24: max relative error {rel[inrange].max():.3e} for |x| <= 6, "
          f"{rel.max():.3e} over [-30, 6]")
    assert np.all(rel <= (2.0 + 1.2 * np.abs(x.astype(np.float64))) * 2.0 ** -23)
    assert rel[inrange].max() <= 1.1e-6


def test_angle_tile_atan2():
    """The angle-storage tile's atan2 (octant reduction, the minimax
    polynomial of atan_poly.cuh, no division) against FP64 atan2: random
    pairs over eight decades of magnitude and both signs, the circle at
    2 million angles (every octant boundary), the axes and the diagonals.
    Bound: the polynomial's 6e-9, the quotient's and the evaluation's FP32
    roundings (a few ulp of an angle below pi/4) and the final pi/2 - a and
    pi - a (half an ulp of pi, with the constants' remainders added back):
    4e-7 rad, below the 3 ulp (7.2e-7) of atan2f that the over-relaxation
    bound of the angle kind allows for."""
    from paper_1211_0780_b300 import xy
    rng = np.random.default_rng(11)
    n = 1 << 22
    x = rng.standard_normal(n) * 10.0 ** rng.uniform(-6, 2, n)
    y = rng.standard_normal(n) * 10.0 ** rng.uniform(-6, 2, n)
    t = np.linspace(-np.pi, np.pi, 2_000_001)
    axes = np.array([[1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1], [-1, 0.0]])
    pts = np.concatenate([np.stack([x, y], 1), 3.7 * np.stack([np.cos(t), np.sin(t)], 1), 2.5 * axes])
    pts = pts.astype(np.float32)
    got = xy.fast_math("atan2", pts).astype(np.float64)
    ref = np.arctan2(pts[:, 1].astype(np.float64), pts[:, 0].astype(np.float64))
    d = np.abs(got - ref)
    d = np.minimum(d, 2 * np.pi - d)
    print(f"\nangle-tile atan2, {len(pts)} pairs: max error {d.max():.3e} rad, rms {np.sqrt(np.mean(d ** 2)):.3e}")
    assert d.max() <= 4e-7
    assert np.all(np.abs(got) <= np.pi + 1e-6)


def test_observable_errors_against_the_oracle():
    """Every record of a measured run (32^3, two replicas, 1 + 2 sweeps, 24
    records each) against the oracle's FP64 sums of the exact angles of the
    stored state it was taken from, then U_L = 1 - <m^4>/(3 <m^2>^2) and
    rho_s = (1/3N) sum_mu (<C_mu> - beta <S_mu^2>) of each replica's series
    from both, and the reweighted U_L, rho_s L and their derivatives of a
    10^5-sample series at 64 couplings against the oracle's FP64 reweighting
    of the same series (relative to the curve's largest magnitude)."""
    from paper_1211_0780_b300 import xy
    from paper_1211_0780_b300.inputs import synthetic_series
    L, R, n = 32, 2, 24
    N = L ** 3
    betas = [0.4542, 0.4560]
    s = xy.Simulation(L, R, betas, SEED, series_capacity=n + 1)
    s.sweep(1, 2, 10)
    gpu, ref = [], []
    for _ in range(n):
        s.sweep(1, 2, 1, measure_every=1)
        rec = s.read_series()
        for slot, th in enumerate(stored_angles64(s)):
            o = oracle.measure(th)
            r = rec[rec["slot"] == slot][0]
            gpu.append((slot, r["E"], r["Mx"], r["My"], *r["C"], *r["S"]))
            ref.append((slot, o.E, o.Mx, o.My, *o.C, *o.S))
    gpu, ref = np.array(gpu), np.array(ref)
    err = np.abs(gpu - ref)
    rows = [("E per bond", err[:, 1].max() / (3 * N)), ("M per site", err[:, 2:4].max() / N),
            ("C_mu per bond", err[:, 4:7].max() / N), ("S_mu per bond", err[:, 7:10].max() / N)]

    def estimators(a, beta):
        m2 = (a[:, 2] ** 2 + a[:, 3] ** 2) / N ** 2
        U = 1.0 - np.mean(m2 ** 2) / (3.0 * np.mean(m2) ** 2)
        rho = (np.mean(a[:, 4:7].sum(axis=1)) - beta * np.mean((a[:, 7:10] ** 2).sum(axis=1))) / (3 * N)
        return U, rho

    dU = drho = 0.0
    for slot in range(R):
        bsel = gpu[:, 0] == slot
        beta = betas[slot]  # no exchanges: each slot keeps its coupling
        Ug, rg = estimators(gpu[bsel], beta)
        Uo, ro = estimators(ref[bsel], beta)
        dU, drho = max(dU, abs(Ug - Uo) / abs(Uo)), max(drho, abs(rg - ro) / abs(ro))
    rows += [("U_L of a series (relative)", dU), ("rho_s of a series (relative)", drho)]

    T, K = 10 ** 5, 64
    ser = synthetic_series(L, T, 31)
    bp = np.linspace(0.4530, 0.4555, K)
    f = xy.reweight_forward(ser, 0.4542, bp, L)
    _, dobs = xy.reweight_backward(bp, L, f)
    o = oracle.reweight_observables(ser["E"], ser["m2"], ser["m4"], ser["c"].T, ser["s2"].T, 0.4542, bp, L)
    for name, g, r in (("reweighted U_L", f["U"], o["U"]), ("reweighted rho_s L", f["rhoL"], o["rhoL"]),
                       ("reweighted dU_L/dbeta'", dobs[0], o["dU"]),
                       ("reweighted d(rho_s L)/dbeta'", dobs[1], o["drhoL"])):
        g = g.cpu().numpy()
        rows.append((name + " (relative)", float(np.max(np.abs(g - r)) / np.max(np.abs(r)))))
    print("\n| observable | max error vs FP64 oracle |\n|---|---|")
    for name, v in rows:
        print(f"| {name} | {v:.2e} |")
    vals = dict(rows)
    assert vals["E per bond"] < 2e-6 and vals["C_mu per bond"] < 2e-6 and vals["S_mu per bond"] < 2e-6
    assert vals["M per site"] < 1e-6
    assert vals["U_L of a series (relative)"] < 1e-5 and vals["rho_s of a series (relative)"] < 1e-5
    assert vals["reweighted U_L (relative)"] < 1e-10 and vals["reweighted rho_s L (relative)"] < 1e-10
    assert vals["reweighted dU_L/dbeta' (relative)"] < 1e-8
    assert vals["reweighted d(rho_s L)/dbeta' (relative)"] < 1e-8
