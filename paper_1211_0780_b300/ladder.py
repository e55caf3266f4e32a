"""Adaptive parallel-tempering ladder (Sec. II: the temperature set is
chosen so that the exchange acceptance rate does not depend on the
temperature).

:func:`update` is the library's equal-acceptance step (``xy_ladder_update``);
:func:`adapt` alternates runs of sweeps with exchanges on the device and
updates of one ladder from the measured acceptance rates.  Marshalling and
bookkeeping only: the sweeps, exchanges and the update run in the library.
"""

from __future__ import annotations

import numpy as np

from . import xy


def update(betas, acceptance, damping: float = 1.0) -> np.ndarray:
    b = np.ascontiguousarray(np.asarray(betas, dtype=np.float64))
    a = np.ascontiguousarray(np.asarray(acceptance, dtype=np.float64))
    if a.size != b.size - 1:
        raise ValueError("one acceptance rate per neighbouring pair")
    out = np.zeros_like(b)
    xy._check(xy.lib().xy_ladder_update(b.size, xy._ptr(b), xy._ptr(a), float(damping), xy._ptr(out)),
              "xy_ladder_update")
    return out


def attempts(n0: int, n1: int, R: int) -> np.ndarray:
    """Exchange attempts of each pair (k, k+1) over events n0 .. n1-1: event
    n tries the pairs with k = n mod 2, n mod 2 + 2, ... (even/odd
    alternation of the library's exchange step)."""
    k = np.arange(R - 1)
    n_even = (n1 + 1) // 2 - (n0 + 1) // 2   # events with n even in [n0, n1)
    n_odd = (n1 - n0) - n_even
    return np.where(k % 2 == 0, n_even, n_odd).astype(np.int64)


def acceptance(sim, lattice: int, n_metropolis: int, n_overrelax: int, sweeps: int) -> np.ndarray:
    """Runs `sweeps` sweeps with an exchange after each and returns the
    acceptance rate of every neighbouring pair of the ladder over them."""
    R = sim.R[lattice]
    s0 = sum(sim.R[:lattice])
    acc0 = sim.accepts()[1][s0:s0 + R - 1].astype(np.int64)
    n0 = int(sim.counters()[2])
    sim.sweep(n_metropolis, n_overrelax, sweeps, measure_every=0, pt_swap_every=1)
    acc1 = sim.accepts()[1][s0:s0 + R - 1].astype(np.int64)
    n1 = int(sim.counters()[2])
    return (acc1 - acc0) / np.maximum(attempts(n0, n1, R), 1)


def adapt(sim, lattice: int, n_iter: int, sweeps: int, n_metropolis: int = 1, n_overrelax: int = 2,
          damping: float = 0.7):
    """n_iter rounds of: measure the acceptance rates over `sweeps` sweeps,
    then move the ladder towards equal acceptance.  Returns the history
    [(betas, rates)] (the last entry's rates are measured on the final
    ladder)."""
    hist = []
    for _ in range(n_iter):
        b = sim.ladder(lattice)
        a = acceptance(sim, lattice, n_metropolis, n_overrelax, sweeps)
        hist.append((b, a))
        sim.set_betas(lattice, update(b, a, damping))
    b = sim.ladder(lattice)
    hist.append((b, acceptance(sim, lattice, n_metropolis, n_overrelax, sweeps)))
    return hist
