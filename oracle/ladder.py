"""FP64 oracle of the equal-acceptance ladder update -- TEST INFRASTRUCTURE.

Only ``tests/`` may import this module.  Sec. II chooses the temperature
set so that the exchange acceptance rate does not depend on the
temperature.  The update models the energy distributions near a pair as
Gaussians of a common width sigma, for which the exchange acceptance of
Eq. 3 is erfc(Delta beta sigma / 2); it solves each measured rate for
sigma and chooses new widths proportional to 1 / sigma, which makes all
modelled rates equal, keeping the ends of the ladder and moving each width
the fraction `damping` of the way.  Written with scipy's erfcinv.
"""

from __future__ import annotations

import numpy as np
from scipy.special import erfc, erfcinv


def update(betas, acceptance, damping=1.0):
    b = np.asarray(betas, dtype=np.float64)
    a = np.clip(np.asarray(acceptance, dtype=np.float64), 1e-6, 1.0 - 1e-9)
    width = np.diff(b)
    sigma = 2.0 * erfcinv(a) / width          # the Gaussian model, solved per pair
    target = (1.0 / sigma) / np.sum(1.0 / sigma) * (b[-1] - b[0])
    new_width = (1.0 - damping) * width + damping * target
    out = np.concatenate([[b[0]], b[0] + np.cumsum(new_width)])
    out[-1] = b[-1]
    return out


def gaussian_model_acceptance(betas, sigma_of_beta):
    """Exchange acceptance of Eq. 3 for Gaussian energy distributions of
    width sigma(beta) taken at the pair's midpoint: erfc(Delta sigma / 2)."""
    b = np.asarray(betas, dtype=np.float64)
    mid = 0.5 * (b[1:] + b[:-1])
    return erfc(np.diff(b) * sigma_of_beta(mid) / 2.0)
