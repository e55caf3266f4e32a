"""FP64 CPU oracle of the 3D XY Monte Carlo hot path -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never calls it, and it never calls the product path.

The arithmetic lives in ``xy_oracle.c`` (plain C, FP64, optional OpenMP over
the sites of one half-sweep, which is order independent because every site
draws from a counter-based stream).  This module loads it with ``ctypes``,
building it with gcc on first use, and adds:

* :class:`Simulation` -- the sweep schedule (Metropolis passes, then
  over-relaxation passes, measurement, parallel-tempering exchange) across
  replicas and lattices, with the counters the library's header fixes;
* :func:`reweight_observables` -- U_L (Sec. II, Eq. 5) and rho_s L
  (Eq. 6 with the L scaling of Sec. III, Eq. 8) at each beta' and their
  d/dbeta' from the fluctuation formula.

Natural layout everywhere: ``theta[z, y, x]`` (x fastest), FP64 radians.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "xy_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
# A compiled copy of the oracle to load instead (the mutation tests point it
# at copies with a planted mistake); it is used as it is, never rebuilt.
_LIB_OVERRIDE = os.environ.get("XY_ORACLE_LIBRARY")

TAG_INIT = 1
TAG_MET = 2
TAG_PT = 3

_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile ``xy_oracle.c`` into ``liboracle.so`` (gcc, -O2, OpenMP)."""
    if _LIB_OVERRIDE:
        return _LIB_OVERRIDE
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c99", "-o", _LIB, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        L = _lib
        L.xo_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        L.xo_philox4x32_10.restype = None
        L.xo_u01.argtypes = [ctypes.c_uint32]
        L.xo_u01.restype = ctypes.c_double
        L.xo_draw_words.argtypes = [ctypes.c_int] * 3 + [
            ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, _u32p]
        L.xo_draw_words.restype = None
        L.xo_init_uniform.argtypes = [ctypes.c_int] * 3 + [ctypes.c_uint64, ctypes.c_uint32, _f64p]
        L.xo_init_uniform.restype = None
        L.xo_metropolis_half.argtypes = [ctypes.c_int] * 3 + [
            _f64p, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64,
            ctypes.c_int, ctypes.c_void_p]
        L.xo_metropolis_half.restype = ctypes.c_long
        L.xo_overrelax_half.argtypes = [ctypes.c_int] * 3 + [_f64p, ctypes.c_int]
        L.xo_overrelax_half.restype = None
        L.xo_measure.argtypes = [ctypes.c_int] * 3 + [_f64p, _f64p]
        L.xo_measure.restype = None
        L.xo_pt_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int]
        L.xo_pt_uniform.restype = ctypes.c_double
        L.xo_pt_swap.argtypes = [ctypes.c_int, _f64p, _f64p, _i32p, ctypes.c_uint64,
                                 ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p]
        L.xo_pt_swap.restype = ctypes.c_int
        L.xo_run_chain.argtypes = [ctypes.c_int] * 3 + [
            _f64p, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64,
            ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
        L.xo_run_chain.restype = ctypes.c_long
        L.xo_reweight.argtypes = [ctypes.c_long, _f64p, ctypes.c_int, _f64p, ctypes.c_double,
                                  ctypes.c_int, _f64p, _f64p, _f64p, _f64p, _f64p]
        L.xo_reweight.restype = None
    return _lib


def set_threads(n: int) -> None:
    """Set the OpenMP thread count of the oracle's half-sweeps."""
    os.environ["OMP_NUM_THREADS"] = str(int(n))
    try:
        gomp = ctypes.CDLL("libgomp.so.1")
        gomp.omp_set_num_threads(ctypes.c_int(int(n)))
    except OSError:  # pragma: no cover - libgomp ships with gcc
        pass


# --------------------------------------------------------------------------
# Philox4x32-10 and the stream layout
# --------------------------------------------------------------------------

def philox4x32_10(ctr, key) -> np.ndarray:
    """Four 32-bit words of Philox4x32-10 (Salmon et al., SC'11)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().xo_philox4x32_10(c, k, out)
    return out


def u01(w: int) -> float:
    return float(lib().xo_u01(int(w)))


def draw_words(dims, seed: int, slot: int, colour: int, tag: int, count: int) -> np.ndarray:
    """Raw (proposal, accept) words of every site of one colour, in
    natural order of those sites; shape (n_sites_of_colour, 2)."""
    Lx, Ly, Lz = dims
    n = sum(1 for z in range(Lz) for y in range(Ly) for x in range(Lx) if (x + y + z) % 2 == colour)
    out = np.zeros(2 * n, dtype=np.uint32)
    lib().xo_draw_words(Lx, Ly, Lz, seed, slot, colour, tag, count, out)
    return out.reshape(n, 2)


# --------------------------------------------------------------------------
# Lattice operations (natural layout theta[z, y, x], FP64)
# --------------------------------------------------------------------------

def _dims(theta: np.ndarray):
    Lz, Ly, Lx = theta.shape
    return Lx, Ly, Lz


def _check(theta: np.ndarray) -> None:
    if theta.dtype != np.float64 or not theta.flags["C_CONTIGUOUS"] or theta.ndim != 3:
        raise TypeError("theta must be a C-contiguous float64 array of shape (Lz, Ly, Lx)")


def init_uniform(dims, seed: int, slot: int) -> np.ndarray:
    """theta = 2 pi u from the INIT stream (the initial state of a slot)."""
    Lx, Ly, Lz = dims
    th = np.zeros((Lz, Ly, Lx), dtype=np.float64)
    lib().xo_init_uniform(Lx, Ly, Lz, seed, slot, th.reshape(-1))
    return th


def metropolis_half(theta: np.ndarray, beta: float, seed: int, slot: int, mpass: int,
                    colour: int, want_margin: bool = False):
    """One Metropolis half-sweep in place; returns (n_accepted, margin or None).
    margin[z,y,x] = |u - exp(-beta dE)| at the updated sites, +inf elsewhere."""
    _check(theta)
    Lx, Ly, Lz = _dims(theta)
    margin = None
    mptr = None
    if want_margin:
        margin = np.full(theta.shape, np.inf, dtype=np.float64)
        mptr = margin.ctypes.data_as(ctypes.c_void_p)
    acc = lib().xo_metropolis_half(Lx, Ly, Lz, theta.reshape(-1), beta, seed, slot, mpass,
                                   colour, mptr)
    return int(acc), margin


def overrelax_half(theta: np.ndarray, colour: int) -> None:
    """One over-relaxation half-sweep in place (Eq. 2)."""
    _check(theta)
    Lx, Ly, Lz = _dims(theta)
    lib().xo_overrelax_half(Lx, Ly, Lz, theta.reshape(-1), colour)


@dataclass
class Sums:
    """Lattice sums of one configuration (Eqs. 4-6): E, M, C_mu, S_mu."""

    E: float
    Mx: float
    My: float
    C: np.ndarray
    S: np.ndarray
    N: int

    @property
    def m2(self) -> float:
        return (self.Mx ** 2 + self.My ** 2) / self.N ** 2


def run_chain(theta: np.ndarray, beta: float, seed: int, slot: int, mpass0: int,
              n_metropolis: int, n_overrelax: int, n_sweeps: int, measure_every: int = 1):
    """Single-slot chain in C (no exchange).  Returns (n_accepted, series)
    with series[m] = (E, Mx, My, Cx, Cy, Cz, Sx, Sy, Sz) after every
    measure_every-th sweep."""
    _check(theta)
    Lx, Ly, Lz = _dims(theta)
    n_meas = n_sweeps // measure_every if measure_every > 0 else 0
    series = np.zeros((max(n_meas, 1), 9), dtype=np.float64)
    acc = lib().xo_run_chain(Lx, Ly, Lz, theta.reshape(-1), beta, seed, slot, mpass0,
                             n_metropolis, n_overrelax, n_sweeps, measure_every,
                             series.ctypes.data_as(ctypes.c_void_p))
    return int(acc), series[:n_meas]


def measure(theta: np.ndarray) -> Sums:
    _check(theta)
    Lx, Ly, Lz = _dims(theta)
    out = np.zeros(9, dtype=np.float64)
    lib().xo_measure(Lx, Ly, Lz, theta.reshape(-1), out)
    return Sums(E=out[0], Mx=out[1], My=out[2], C=out[3:6].copy(), S=out[6:9].copy(),
                N=Lx * Ly * Lz)


def pt_uniform(seed: int, ladder: int, count: int, k: int) -> float:
    return float(lib().xo_pt_uniform(seed, ladder, count, k))


def pt_swap(betas, E_by_slot, perm, seed: int, ladder: int, count: int, parity: int):
    """Eq. (3) on one ladder; perm (int32, beta index -> slot) is updated in
    place.  Returns (n_accepted, accepted-per-pair int32 array)."""
    b = np.ascontiguousarray(betas, dtype=np.float64)
    e = np.ascontiguousarray(E_by_slot, dtype=np.float64)
    if perm.dtype != np.int32 or not perm.flags["C_CONTIGUOUS"]:
        raise TypeError("perm must be C-contiguous int32")
    acc = np.zeros(len(b), dtype=np.int32)
    n = lib().xo_pt_swap(len(b), b, e, perm, seed, ladder, count, parity,
                         acc.ctypes.data_as(ctypes.c_void_p))
    return int(n), acc


# --------------------------------------------------------------------------
# Sweep schedule over lattices and replicas
# --------------------------------------------------------------------------

@dataclass
class Record:
    """One measurement of one slot."""

    sweep: int
    slot: int
    beta_index: int
    beta: float
    sums: Sums


@dataclass
class Simulation:
    """Replicas of cubic (or Lx x Ly x Lz) lattices under the sweep schedule.

    Slots are numbered globally: lattice 0's replicas first.  ``perm[l][k]``
    is the slot (local to lattice l) at the k-th beta of that lattice's
    ascending ladder.  Counters: ``mpass`` counts Metropolis passes (a pass
    is one black and one white half-sweep), ``sweep`` counts sweeps and
    ``nswap`` counts exchange events; each sits in the Philox counter of its
    stream, so every draw is a pure function of (seed, counter, slot, site).
    """

    dims: list
    betas: list
    seed: int
    theta: list = field(default_factory=list)
    perm: list = field(default_factory=list)
    mpass: int = 0
    sweep: int = 0
    nswap: int = 0
    records: list = field(default_factory=list)
    swap_accepts: list = field(default_factory=list)

    @classmethod
    def create(cls, Ls, n_replicas, betas, seed: int):
        dims, blist, theta, perm = [], [], [], []
        slot = 0
        off = 0
        for L, R in zip(Ls, n_replicas):
            d = tuple(L) if isinstance(L, (tuple, list)) else (L, L, L)
            dims.append(d)
            b = np.asarray(betas[off:off + R], dtype=np.float64)
            off += R
            blist.append(b)
            for _ in range(R):
                theta.append(init_uniform(d, seed, slot))
                slot += 1
            perm.append(np.arange(R, dtype=np.int32))
        sim = cls(dims=dims, betas=blist, seed=seed, theta=theta, perm=perm)
        sim.swap_accepts = [np.zeros(len(b), dtype=np.int64) for b in blist]
        return sim

    def slots(self):
        """Yield (lattice, local replica, global slot)."""
        g = 0
        for l, b in enumerate(self.betas):
            for r in range(len(b)):
                yield l, r, g
                g += 1

    def beta_of(self, l: int, r: int) -> float:
        k = int(np.nonzero(self.perm[l] == r)[0][0])
        return float(self.betas[l][k])

    def metropolis_pass(self):
        for l, r, g in self.slots():
            beta = self.beta_of(l, r)
            for c in (0, 1):
                metropolis_half(self.theta[g], beta, self.seed, g, self.mpass, c)
        self.mpass += 1

    def overrelax_pass(self):
        for _, _, g in self.slots():
            for c in (0, 1):
                overrelax_half(self.theta[g], c)

    def exchange(self, parity: int | None = None):
        """One exchange event on every ladder; energies measured afresh."""
        par = (self.nswap & 1) if parity is None else parity
        total = 0
        for l, b in enumerate(self.betas):
            base = sum(len(x) for x in self.betas[:l])
            E = np.array([measure(self.theta[base + r]).E for r in range(len(b))])
            n, acc = pt_swap(b, E, self.perm[l], self.seed, l, self.nswap, par)
            self.swap_accepts[l] += acc
            total += n
        self.nswap += 1
        return total

    def run(self, n_metropolis: int, n_overrelax: int, n_sweeps: int,
            measure_every: int = 0, pt_swap_every: int = 0):
        """Sweeps in the library's order: n_metropolis Metropolis passes,
        n_overrelax over-relaxation passes, then (if due) the measurement of
        every slot and (if due) one exchange event per ladder."""
        for _ in range(n_sweeps):
            for _ in range(n_metropolis):
                self.metropolis_pass()
            for _ in range(n_overrelax):
                self.overrelax_pass()
            s = self.sweep
            if measure_every > 0 and (s + 1) % measure_every == 0:
                for l, r, g in self.slots():
                    k = int(np.nonzero(self.perm[l] == r)[0][0])
                    self.records.append(Record(sweep=s, slot=g, beta_index=k,
                                               beta=float(self.betas[l][k]),
                                               sums=measure(self.theta[g])))
            if pt_swap_every > 0 and (s + 1) % pt_swap_every == 0:
                self.exchange()
            self.sweep += 1


# --------------------------------------------------------------------------
# Single-histogram reweighting
# --------------------------------------------------------------------------

def reweight(E, O, beta0: float, betap):
    """FP64 reweighting of columns O[t, j] measured at beta0 with energies
    E[t] to each beta'_k.  Returns (logZ[K], meanE[K], mean[K, n], cov[K, n])
    with cov = <O E> - <O><E> (so d<O>/dbeta' = -cov)."""
    E = np.ascontiguousarray(E, dtype=np.float64)
    O = np.ascontiguousarray(O, dtype=np.float64)
    if O.ndim == 1:
        O = O[:, None]
    T, n = O.shape
    bp = np.ascontiguousarray(betap, dtype=np.float64)
    K = len(bp)
    logZ = np.zeros(K)
    meanE = np.zeros(K)
    mean = np.zeros((K, n))
    cov = np.zeros((K, n))
    lib().xo_reweight(T, E, n, O.reshape(-1), float(beta0), K, bp, logZ, meanE,
                      mean.reshape(-1), cov.reshape(-1))
    return logZ, meanE, mean, cov


def reweight_observables(E, m2, m4, c, s2, beta0: float, betap, L: int):
    """Binder ratio U_L = 1 - <m^4>/(3 <m^2>^2) (Eq. 5) and rho_s L, with
    rho_s = (1/3) sum_mu (<c_mu> - beta' <s2_mu>) (Eq. 6, columns normalised
    by N: c_mu = C_mu / N, s2_mu = S_mu^2 / N), at each beta', and both
    derivatives d/dbeta' by the chain rule on d<O>/dbeta' = -cov(O, E).

    c and s2 are (T, 3) arrays; m2, m4 are (T,).  Returns a dict of FP64
    arrays of length K."""
    csum = np.asarray(c, dtype=np.float64).sum(axis=1)
    s2sum = np.asarray(s2, dtype=np.float64).sum(axis=1)
    O = np.stack([np.asarray(m2, np.float64), np.asarray(m4, np.float64), csum, s2sum], axis=1)
    bp = np.asarray(betap, dtype=np.float64)
    logZ, meanE, mean, cov = reweight(E, O, beta0, bp)
    mm2, mm4, mc, ms2 = mean.T
    d2, d4, dc, ds2 = (-cov).T
    U = 1.0 - mm4 / (3.0 * mm2 ** 2)
    dU = -(d4 / (3.0 * mm2 ** 2) - 2.0 * mm4 * d2 / (3.0 * mm2 ** 3))
    rhoL = L / 3.0 * (mc - bp * ms2)
    drhoL = L / 3.0 * (dc - ms2 - bp * ds2)
    return {"logZ": logZ, "E": meanE, "m2": mm2, "m4": mm4, "c": mc, "s2": ms2,
            "U": U, "rhoL": rhoL, "dU": dU, "drhoL": drhoL}
