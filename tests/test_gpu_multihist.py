"""Multi-histogram reweighting kernels vs the FP64 oracle."""

import numpy as np
import pytest

import oracle
from oracle import multihist as omh

pytestmark = pytest.mark.gpu


def _ladder_series(betas, n, L, seed):
    """Per-coupling synthetic series: Gaussian energies of a Gaussian density
    of states (E0 - beta s^2, width s) with observables correlated with E."""
    rng = np.random.default_rng(seed)
    N = L ** 3
    E0, s = -1.2 * N, 1.5 * np.sqrt(N)
    out = []
    for b in betas:
        E = E0 - b * s * s + s * rng.standard_normal(n)
        z = (E - E.mean()) / s
        m2 = np.clip(0.05 * rng.gamma(4.0, 0.25, n) * np.exp(-0.3 * z), 0, 1)
        c = np.tile(-E / (3 * N), (3, 1)) + 0.01 * rng.standard_normal((3, n))
        S = np.sqrt(0.3 * N) * rng.standard_normal((3, n))
        out.append({"E": E, "m2": m2.astype(np.float32), "m4": (m2 * m2).astype(np.float32),
                    "c": c.astype(np.float32), "s2": (S * S / N).astype(np.float32)})
    return out


def _oracle_outputs(pooled, betas, counts, f, bp, L):
    O = np.stack([pooled["m2"].astype(np.float64), pooled["m4"].astype(np.float64),
                  pooled["c"].astype(np.float64).sum(axis=0), pooled["s2"].astype(np.float64).sum(axis=0)], axis=1)
    mE, mO, cov = omh.averages(pooled["E"], O, betas, counts, f, bp)
    m2, m4, c, s2 = mO.T
    return {"E": mE, "m2": m2, "m4": m4, "csum": c, "s2sum": s2, "U": 1 - m4 / (3 * m2 * m2), "q2": m4 / (m2 * m2),
            "rhoL": L / 3 * (c - np.asarray(bp) * s2), "cov_m2": cov[:, 0], "cov_m4": cov[:, 1]}


@pytest.mark.parametrize("R,n", [(8, 4000), (3, 7001)])
def test_solve_and_forward_match_oracle(R, n):
    from paper_1211_0780_b300 import multihist as mh
    L = 16
    betas = np.linspace(0.44, 0.47, R)
    pooled, counts = mh.pool(_ladder_series(betas, n, L, 5 + R))
    f, it = mh.solve(pooled, betas, counts, tol=1e-12)
    fo, ito = omh.solve(pooled["E"], betas, counts, tol=1e-13)
    np.testing.assert_allclose(f, fo, atol=1e-9)
    assert it > 1
    bp = np.linspace(0.438, 0.472, 41)
    g = mh.forward(pooled, betas, counts, f, bp, L)
    ref = _oracle_outputs(pooled, betas, counts, fo, bp, L)
    for key in ("E", "m2", "m4", "U", "rhoL", "q2"):
        np.testing.assert_allclose(g[key].cpu().numpy(), ref[key], rtol=1e-9, err_msg=key)
    np.testing.assert_allclose(g["cov_m2"].cpu().numpy(), ref["cov_m2"], rtol=1e-7,
                               atol=1e-9 * np.max(np.abs(ref["cov_m2"])))


def test_one_coupling_equals_single_histogram_kernels():
    from paper_1211_0780_b300 import multihist as mh, xy
    L = 24
    s = _ladder_series([0.4542], 9000, L, 3)[0]
    pooled, counts = mh.pool([s])
    f, _ = mh.solve(pooled, [0.4542], counts)
    bp = np.linspace(0.4500, 0.4590, 37)
    g = mh.forward(pooled, [0.4542], counts, f, bp, L)
    r = xy.reweight_forward(pooled, 0.4542, bp, L)
    for key in ("E", "m2", "m4", "csum", "s2sum", "U", "rhoL", "q2"):
        np.testing.assert_allclose(g[key].cpu().numpy(), r[key].cpu().numpy(), rtol=1e-10, err_msg=key)


def test_simulated_ladder_matches_oracle():
    """Records of the library's own parallel-tempering run, split by beta
    index: the pooled estimate agrees with the oracle's."""
    from paper_1211_0780_b300 import multihist as mh, xy
    L, R = 8, 5
    betas = np.linspace(0.43, 0.48, R)
    sim = xy.Simulation(L, R, betas, 17, series_capacity=3000)
    sim.sweep(1, 2, 300, pt_swap_every=1)
    sim.read_series()
    sim.sweep(1, 2, 3000, measure_every=1, pt_swap_every=1)
    parts, b = mh.series_from_records(sim.read_series(), L, R)
    np.testing.assert_allclose(b, betas)
    pooled, counts = mh.pool(parts)
    f, _ = mh.solve(pooled, b, counts, tol=1e-12)
    fo, _ = omh.solve(pooled["E"], b, counts, tol=1e-13)
    np.testing.assert_allclose(f, fo, atol=1e-9)
    bp = np.linspace(0.43, 0.48, 26)
    g = mh.forward(pooled, b, counts, f, bp, L)
    ref = _oracle_outputs(pooled, b, counts, fo, bp, L)
    for key in ("E", "U", "rhoL"):
        np.testing.assert_allclose(g[key].cpu().numpy(), ref[key], rtol=1e-9, err_msg=key)


def test_iteration_cap_reports_timeout():
    from paper_1211_0780_b300 import multihist as mh, xy
    betas = np.linspace(0.44, 0.47, 4)
    pooled, counts = mh.pool(_ladder_series(betas, 2000, 8, 1))
    with pytest.raises(xy.XYError) as e:
        mh.solve(pooled, betas, counts, tol=1e-14, max_iter=1)
    assert e.value.status == xy.XY_ERR_TIMEOUT
