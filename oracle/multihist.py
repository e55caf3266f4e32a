"""FP64 oracle of multi-histogram reweighting -- TEST INFRASTRUCTURE.

Only ``tests/`` may import this module; the product path never calls it.
Ferrenberg and Swendsen's multiple-histogram equations written out with
numpy/scipy log-sum-exp, in their textbook form: the records of R couplings
pooled, N_m records measured at beta_m,

    f_k = -log sum_t exp(-beta_k E_t) / sum_m N_m exp(f_m - beta_m E_t),

iterated to a fixed point (normalised f_0 = 0), and

    <O>_beta = sum_t O_t w_t(beta) / sum_t w_t(beta),
    w_t(beta) = exp(-beta E_t) / sum_m N_m exp(f_m - beta_m E_t).
"""

from __future__ import annotations

import numpy as np
from scipy.special import logsumexp


def log_denominator(E, betas, counts, f):
    a = np.log(np.asarray(counts, np.float64))[None, :] + np.asarray(f)[None, :] \
        - np.asarray(E, np.float64)[:, None] * np.asarray(betas, np.float64)[None, :]
    return logsumexp(a, axis=1)


def solve(E, betas, counts, tol=1e-12, max_iter=100000):
    E = np.asarray(E, np.float64)
    b = np.asarray(betas, np.float64)
    f = np.zeros(len(b))
    for it in range(max_iter):
        lD = log_denominator(E, b, counts, f)
        fn = -logsumexp(-b[None, :] * E[:, None] - lD[:, None], axis=0)
        fn -= fn[0]
        if np.max(np.abs(fn - f)) <= tol:
            return fn, it + 1
        f = fn
    return f, max_iter


def averages(E, O, betas, counts, f, betap):
    """<O_j> and cov(O_j, E) at each beta' (O: [T, n])."""
    E = np.asarray(E, np.float64)
    O = np.asarray(O, np.float64)
    lD = log_denominator(E, betas, counts, f)
    out_mean, out_E, out_cov = [], [], []
    for bp in np.atleast_1d(betap):
        lw = -bp * E - lD
        w = np.exp(lw - lw.max())
        w /= w.sum()
        mE = w @ E
        mO = w @ O
        out_E.append(mE)
        out_mean.append(mO)
        out_cov.append(w @ (O * E[:, None]) - mO * mE)
    return np.array(out_E), np.array(out_mean), np.array(out_cov)
