"""Adaptive ladder (Sec. II: equal exchange acceptance): the oracle's update
pinned on the Gaussian acceptance model, and the library's update (host
code, no GPU needed) against the oracle."""

import numpy as np
import pytest
from scipy.special import erfc

from oracle import ladder as olad


def test_constant_width_gives_equal_spacing_in_one_step():
    """With sigma independent of beta the equal-acceptance ladder is evenly
    spaced; one full update reaches it from any ladder."""
    b = np.array([0.40, 0.41, 0.45, 0.46, 0.47, 0.55])
    sig = lambda x: np.full_like(x, 40.0)
    new = olad.update(b, olad.gaussian_model_acceptance(b, sig), 1.0)
    np.testing.assert_allclose(np.diff(new), np.full(5, 0.03), rtol=1e-12)
    a = olad.gaussian_model_acceptance(new, sig)
    assert np.ptp(a) < 1e-12


def test_iteration_equalises_acceptance_for_constant_heat_capacity():
    """sigma_E^2 = C / beta^2 (constant heat capacity): iterating the update
    drives every modelled acceptance to the same value, and that ladder is
    close to geometric (equal ratios beta_k+1 / beta_k)."""
    b = np.linspace(0.2, 0.8, 12)
    sig = lambda x: np.sqrt(400.0) / x
    for _ in range(40):
        b = olad.update(b, olad.gaussian_model_acceptance(b, sig), 0.8)
    a = olad.gaussian_model_acceptance(b, sig)
    assert np.ptp(a) < 1e-9 * a.mean()
    r = b[1:] / b[:-1]
    assert np.ptp(r) < 1e-3


def test_fixed_point_ends_and_damping():
    b = np.array([0.30, 0.34, 0.39, 0.45])
    same = olad.update(b, [0.4, 0.4, 0.4], 1.0)
    np.testing.assert_allclose(same, b, rtol=0, atol=1e-15)
    moved = olad.update(b, [0.9, 0.1, 0.5], 1.0)
    assert moved[0] == b[0] and moved[-1] == b[-1] and np.all(np.diff(moved) > 0)
    np.testing.assert_array_equal(olad.update(b, [0.9, 0.1, 0.5], 0.0), b)
    # a pair that accepts more gets wider
    assert np.diff(moved)[0] > np.diff(b)[0] and np.diff(moved)[1] < np.diff(b)[1]


def test_library_update_matches_oracle():
    from paper_1211_0780_b300 import ladder
    rng = np.random.default_rng(3)
    for R in (2, 3, 8, 32):
        for damping in (1.0, 0.5, 0.0):
            b = np.sort(rng.uniform(0.3, 0.6, R))
            a = rng.uniform(0.0, 1.0, R - 1)
            a[0] = 0.0 if R > 2 else a[0]
            np.testing.assert_allclose(ladder.update(b, a, damping), olad.update(b, a, damping),
                                       rtol=1e-12, atol=1e-14)


def test_library_update_rejects_bad_input():
    from paper_1211_0780_b300 import ladder, xy
    with pytest.raises(xy.XYError):
        ladder.update([0.5, 0.4], [0.3])
    with pytest.raises(xy.XYError):
        ladder.update([0.4, 0.5], [1.3])
    with pytest.raises(xy.XYError):
        ladder.update([0.4, 0.5], [0.3], damping=1.5)


def test_attempt_count():
    from paper_1211_0780_b300.ladder import attempts
    # events 3, 4, 5, 6: even events 4, 6 try pairs 0, 2; odd 3, 5 try 1, 3
    np.testing.assert_array_equal(attempts(3, 7, 5), [2, 2, 2, 2])
    np.testing.assert_array_equal(attempts(0, 5, 4), [3, 2, 3])
