"""Seeded synthetic inputs shared by the tests, the smoke check and the
benchmark.  This module holds random-number generation only -- none of the
method's arithmetic -- so that the CUDA path and the oracle can be fed the
same inputs without sharing code.

* :func:`random_angles` -- i.i.d. angles uniform in [0, 2pi) (a hot start);
* :func:`synthetic_series` -- a measurement series shaped like one from an
  L^3 run near beta_c = 0.4542 (the critical coupling the paper's crossings
  locate, T_c ~ 2.2018): Gaussian total energy with the scale of an
  equilibrium series (mean -0.99 N, standard deviation 2.2 sqrt(N)), a
  Gamma-distributed |m|^2 anti-correlated with E, |m|^4 = (|m|^2)^2, bond
  cosines c_mu = C_mu / N consistent with E (sum_mu c_mu = -E/N), and
  s2_mu = S_mu^2 / N from Gaussian S_mu.  Used to time reweighting and to
  test it; statistics of real runs are not needed for either.
"""

from __future__ import annotations

import numpy as np


def random_angles(shape, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 2.0 * np.pi, size=shape).astype(np.float64)


def synthetic_series(L: int, T: int, seed: int) -> dict:
    rng = np.random.default_rng(seed)
    N = L ** 3
    z = rng.standard_normal(T)
    E = -0.99 * N + 2.2 * np.sqrt(N) * z
    k = 4.1
    mu2 = 0.8 * float(L) ** -1.04
    a = 0.3
    m2 = mu2 * rng.gamma(k, 1.0 / k, size=T) * np.exp(-a * z - 0.5 * a * a)
    m2 = np.clip(m2, 0.0, 1.0)
    eta = 0.01 * rng.standard_normal((3, T))
    eta -= eta.mean(axis=0, keepdims=True)
    c = (-E / (3.0 * N))[None, :] + eta
    S = np.sqrt(0.3 * N) * rng.standard_normal((3, T))
    s2 = S * S / N
    return {
        "E": E.astype(np.float64),
        "m2": m2.astype(np.float32),
        "m4": (m2 * m2).astype(np.float32),
        "c": c.astype(np.float32),
        "s2": s2.astype(np.float32),
        "L": L,
        "N": N,
    }
