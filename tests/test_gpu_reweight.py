"""Reweighting kernels (forward, backward, autograd) vs the FP64 oracle."""

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def _series(L, T, seed):
    from paper_1211_0780_b300.inputs import synthetic_series
    return synthetic_series(L, T, seed)


def _oracle(s, beta0, bp, L):
    return oracle.reweight_observables(s["E"], s["m2"], s["m4"], s["c"].T, s["s2"].T, beta0, bp, L)


@pytest.mark.parametrize("L,T,K", [(8, 5000, 37), (32, 20000, 300), (64, 3000, 1025)])
def test_forward_backward_match_oracle(L, T, K):
    """All outputs and derivatives agree with the oracle to 1e-8 relative."""
    from paper_1211_0780_b300 import xy
    s = _series(L, T, 7 + L)
    beta0 = 0.4542
    bp = np.linspace(0.4530, 0.4555, K)
    f = xy.reweight_forward(s, beta0, bp, L)
    _, dobs = xy.reweight_backward(bp, L, f)
    ref = _oracle(s, beta0, bp, L)
    for key, gk in (("logZ", "logZ"), ("E", "E"), ("m2", "m2"), ("m4", "m4"), ("U", "U"), ("rhoL", "rhoL")):
        np.testing.assert_allclose(f[gk].cpu().numpy(), ref[key], rtol=1e-10, err_msg=key)
    # q2 = <m^4>/<m^2>^2 of the collapse (Eq. 11), from the oracle's moments
    np.testing.assert_allclose(f["q2"].cpu().numpy(), ref["m4"] / ref["m2"] ** 2, rtol=1e-10)
    # Relative to each curve's scale: dU/dbeta' crosses zero inside the grid.
    for row, key in ((0, "dU"), (1, "drhoL")):
        np.testing.assert_allclose(dobs[row].cpu().numpy(), ref[key], rtol=1e-8,
                                   atol=1e-8 * np.max(np.abs(ref[key])))
    # dq2/dbeta' = -3 dU/dbeta' (Eq. 11: q2 = 3 (1 - U_L))
    np.testing.assert_allclose(dobs[2].cpu().numpy(), -3.0 * ref["dU"], rtol=1e-8,
                               atol=3e-8 * np.max(np.abs(ref["dU"])))


def test_non_uniform_grid_and_sign_change():
    """Unevenly spaced beta' (no stepping) and a grid crossing beta0."""
    from paper_1211_0780_b300 import xy
    L, T = 16, 4000
    s = _series(L, T, 3)
    bp = np.sort(np.random.default_rng(1).uniform(0.4500, 0.4580, 61))
    f = xy.reweight_forward(s, 0.4542, bp, L)
    ref = _oracle(s, 0.4542, bp, L)
    np.testing.assert_allclose(f["logZ"].cpu().numpy(), ref["logZ"], rtol=1e-11)
    np.testing.assert_allclose(f["U"].cpu().numpy(), ref["U"], rtol=1e-10)
    np.testing.assert_allclose(f["rhoL"].cpu().numpy(), ref["rhoL"], rtol=1e-10)


def test_identity_at_beta0():
    from paper_1211_0780_b300 import xy
    s = _series(8, 3000, 5)
    f = xy.reweight_forward(s, 0.4542, np.array([0.4542, 0.4542]), 8)
    assert f["logZ"][0].item() == pytest.approx(np.log(3000), rel=1e-13)
    assert f["m2"][0].item() == pytest.approx(float(s["m2"].astype(np.float64).mean()), rel=1e-13)


def test_autograd_matches_finite_differences_and_fluctuation_formula():
    """d/dbeta' through torch.autograd equals the fluctuation formula to 1e-8
    and a central difference of the forward kernel (h = 1e-7) to 1e-6."""
    import torch
    from paper_1211_0780_b300 import xy
    L, T, K = 32, 20000, 64
    s = _series(L, T, 11)
    bp = torch.linspace(0.4530, 0.4555, K, dtype=torch.float64, device="cuda", requires_grad=True)
    U, R = xy.reweight(s, 0.4542, bp, L)
    (U.sum() + 2.0 * R.sum()).backward()
    g = bp.grad.cpu().numpy()
    ref = _oracle(s, 0.4542, bp.detach().cpu().numpy(), L)
    want = ref["dU"] + 2.0 * ref["drhoL"]
    np.testing.assert_allclose(g, want, rtol=1e-8, atol=1e-8 * np.max(np.abs(want)))
    h = 1e-7
    b = bp.detach()
    fp = xy.reweight_forward(s, 0.4542, b + h, L)
    fm = xy.reweight_forward(s, 0.4542, b - h, L)
    fd = ((fp["U"] - fm["U"]) + 2.0 * (fp["rhoL"] - fm["rhoL"])).cpu().numpy() / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-6 * np.max(np.abs(fd)))


@pytest.mark.parametrize("T", [2, 777])
def test_constant_energy_series_closed_forms(T):
    """A series whose energy never changes (the shortest series the call
    accepts, two samples, and a longer one):
    every weight is the same, so at any beta' the averages are the plain
    means, log Z = log T - (beta' - beta0) E0, the covariances with E vanish,
    dU_L/dbeta' = 0 and d(rho_s L)/dbeta' = -(L/3) <s2> (the explicit beta'
    of Eq. 6 alone)."""
    from paper_1211_0780_b300 import xy
    rng = np.random.default_rng(T)
    L, beta0, E0 = 8, 0.4542, -1234.5
    m2 = rng.random(T).astype(np.float32)
    s = {"E": np.full(T, E0), "m2": m2, "m4": (m2 * m2).astype(np.float32),
         "c": rng.random((3, T)).astype(np.float32), "s2": rng.random((3, T)).astype(np.float32)}
    bp = np.array([0.440, beta0, 0.470])
    f = xy.reweight_forward(s, beta0, bp, L)
    m2m = s["m2"].astype(np.float64).mean()
    m4m = s["m4"].astype(np.float64).mean()
    cm = s["c"].astype(np.float64).sum(axis=0).mean()
    s2m = s["s2"].astype(np.float64).sum(axis=0).mean()
    for k, b in enumerate(bp):
        assert f["logZ"][k].item() == pytest.approx(np.log(T) - (b - beta0) * E0, rel=1e-12, abs=1e-9)
        assert f["E"][k].item() == pytest.approx(E0, rel=1e-14)
        assert f["m2"][k].item() == pytest.approx(m2m, rel=1e-12)
        assert f["m4"][k].item() == pytest.approx(m4m, rel=1e-12)
        assert f["csum"][k].item() == pytest.approx(cm, rel=1e-12)
        assert f["s2sum"][k].item() == pytest.approx(s2m, rel=1e-12)
        assert f["U"][k].item() == pytest.approx(1.0 - m4m / (3.0 * m2m * m2m), rel=1e-12)
        assert f["rhoL"][k].item() == pytest.approx(L / 3.0 * (cm - b * s2m), rel=1e-12)
        for name in xy.COV_ROWS:
            assert abs(f["cov_" + name][k].item()) <= 1e-12
    _, dobs = xy.reweight_backward(bp, L, f)
    d = dobs.cpu().numpy()
    np.testing.assert_allclose(d[0], 0.0, atol=1e-12)
    np.testing.assert_allclose(d[1], -L / 3.0 * s2m, rtol=1e-12)


def test_one_sample_series_is_rejected():
    """T < 2 is an argument error (nothing is computed)."""
    from paper_1211_0780_b300 import xy
    s = {"E": np.array([-1.0]), "m2": np.ones(1, np.float32), "m4": np.ones(1, np.float32),
         "c": np.ones((3, 1), np.float32), "s2": np.ones((3, 1), np.float32)}
    with pytest.raises(xy.XYError) as e:
        xy.reweight_forward(s, 0.4542, np.array([0.45]), 8)
    assert e.value.status == xy.XY_ERR_ARG
