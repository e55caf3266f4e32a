"""Pins of the multi-histogram oracle (CPU): reduction to single-histogram
reweighting for one coupling, exact free energies and energies of a
Gaussian density of states (equal and unequal record counts), and the
energy-shift covariance."""

import numpy as np
import pytest

import oracle
from oracle import multihist as omh


def _gaussian_ladder(betas, n, E0, s, seed):
    """Exact canonical samples of g(E) ~ exp(-(E - E0)^2 / (2 s^2)): at beta
    they are Gaussian with mean E0 - beta s^2 and width s."""
    rng = np.random.default_rng(seed)
    return [E0 - b * s * s + s * rng.standard_normal(n) for b in betas]


def test_one_coupling_is_single_histogram_reweighting():
    rng = np.random.default_rng(1)
    E = -3000 + 40 * rng.standard_normal(5000)
    O = np.stack([rng.gamma(3, 1, 5000) + 0.001 * E, np.sin(E)], axis=1)
    f, _ = omh.solve(E, [0.45], [5000])
    bp = np.linspace(0.44, 0.46, 7)
    mE, mO, cov = omh.averages(E, O, [0.45], [5000], f, bp)
    _, rE, rO, rcov = oracle.reweight(E, O, 0.45, bp)
    np.testing.assert_allclose(mE, rE, rtol=1e-12)
    np.testing.assert_allclose(mO, rO, rtol=1e-10)
    np.testing.assert_allclose(cov, rcov, rtol=1e-8, atol=1e-10)


def test_gaussian_density_of_states():
    """f_k - f_0 = -(ln Z_k - ln Z_0) with ln Z(beta) = -beta E0 + beta^2 s^2 / 2,
    and <E>(beta') = E0 - beta' s^2 between the couplings (statistical)."""
    betas = np.linspace(0.40, 0.50, 6)
    E0, s, n = -2000.0, 30.0, 20000
    parts = _gaussian_ladder(betas, n, E0, s, 7)
    E = np.concatenate(parts)
    f, it = omh.solve(E, betas, [n] * 6, tol=1e-11)
    lnZ = -betas * E0 + betas ** 2 * s * s / 2
    np.testing.assert_allclose(f, -(lnZ - lnZ[0]), atol=0.05)
    bp = np.linspace(0.41, 0.49, 9)
    mE, _, cov = omh.averages(E, E[:, None], betas, [n] * 6, f, bp)
    np.testing.assert_allclose(mE, E0 - bp * s * s, atol=0.05 * s)
    np.testing.assert_allclose(cov[:, 0], s * s, rtol=0.05)  # the variance of E is s^2


def test_energy_shift():
    betas = np.array([0.42, 0.45, 0.48])
    E = np.concatenate(_gaussian_ladder(betas, 3000, -1000.0, 20.0, 3))
    f, _ = omh.solve(E, betas, [3000] * 3)
    g, _ = omh.solve(E + 123.0, betas, [3000] * 3)
    np.testing.assert_allclose(g, f + (betas - betas[0]) * 123.0, atol=1e-8)
    bp = [0.43, 0.47]
    a = omh.averages(E, E[:, None], betas, [3000] * 3, f, bp)[0]
    b = omh.averages(E + 123.0, E[:, None], betas, [3000] * 3, g, bp)[0]
    np.testing.assert_allclose(b, a + 123.0, rtol=1e-12)


def test_unequal_record_counts():
    """Runs with 2,000 and 24,000 records alternating: the counts N_m weight
    each run's histogram, so the exact free energies and energies of the
    Gaussian density of states still come out (statistical)."""
    betas = np.linspace(0.40, 0.50, 6)
    E0, s = -2000.0, 30.0
    ns = [2000, 24000] * 3
    rng = np.random.default_rng(11)
    E = np.concatenate([E0 - b * s * s + s * rng.standard_normal(n) for b, n in zip(betas, ns)])
    f, _ = omh.solve(E, betas, ns, tol=1e-11)
    lnZ = -betas * E0 + betas ** 2 * s * s / 2
    np.testing.assert_allclose(f, -(lnZ - lnZ[0]), atol=0.05)
    bp = np.linspace(0.41, 0.49, 9)
    mE, _, cov = omh.averages(E, E[:, None], betas, ns, f, bp)
    np.testing.assert_allclose(mE, E0 - bp * s * s, atol=0.05 * s)
    np.testing.assert_allclose(cov[:, 0], s * s, rtol=0.05)
