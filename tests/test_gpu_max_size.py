"""The largest lattice the library takes, L = 1024 (1.07 G sites, 8.6 GB of
(cos, sin) state): one sweep and one over-relaxation half-sweep on the direct
tile, checked on sampled outputs the oracle computes one by one, and the
fused lattice sums against an FP64 sum over the whole lattice.

Sampled over-relaxation (Eq. 2): for each sampled site the oracle reflects
the spin at the centre of the 4 x 4 x 4 block around it (all six neighbours
inside the block, so its update is the full lattice's), given the exact
angles of the stored vectors; tolerance as in test_gpu_parity.  The
Metropolis half-sweep is checked for what holds at any size: only the
swept colour changes, and every changed site takes the proposal angle
2 pi u0 of its Philox word (within the fast sincos error), which the test
draws with the oracle's Philox4x32-10 at the sampled sites.
"""

import numpy as np
import pytest

import oracle
from helpers import circ_dist

pytestmark = pytest.mark.gpu

SEED = 0x5EED2012
L = 1024
OR_A, OR_B = 8.4e-6, 1e-6   # the conditioning bound of test_gpu_parity
BOND_TOL, SITE_TOL = 2e-6, 1e-6


def packed_index(x, y, z):
    """Index of the cosine of site (x, y, z) of slot 0 in the packed state;
    the sine is N/2 further."""
    N = L ** 3
    return ((x + y + z) % 2) * N + (x >> 1) + (L // 2) * (y + L * z)


def angles_at(pk, x, y, z):
    i = packed_index(x, y, z)
    t = np.arctan2(pk[i + L ** 3 // 2].astype(np.float64), pk[i].astype(np.float64))
    return np.where(t < 0, t + 2 * np.pi, t)


_Y, _X = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
_PLANE = [packed_index(_X, _Y, 0), packed_index(_X, _Y, 1) - (L // 2) * L]  # by the parity of z


def plane_vectors(pk, z):
    """Natural-layout (L, L) FP64 cos and sin of plane z."""
    i = _PLANE[z & 1] + (L // 2) * L * z
    return pk[i].astype(np.float64), pk[i + L ** 3 // 2].astype(np.float64)


def test_largest_lattice_sampled_parity():
    import torch
    from paper_1211_0780_b300 import xy
    if torch.cuda.get_device_properties(0).total_memory < 24 << 30:
        pytest.skip("needs a device with room for a 1024^3 lattice")
    s = xy.Simulation(L, 1, [0.4542], SEED, series_capacity=4)
    s.set_tile(0, 1, 8, 3)
    s.sweep(1, 1, 1)
    rng = np.random.default_rng(5)
    n = 2000

    # over-relaxation of colour 0 on sampled sites
    before = s.get_packed()
    s.overrelax_half(0)
    after = s.get_packed()
    xs, ys, zs = (rng.integers(0, L, 4 * n) for _ in range(3))
    keep = ((xs + ys + zs) % 2) == 0
    xs, ys, zs = xs[keep][:n], ys[keep][:n], zs[keep][:n]
    off = np.arange(-1, 3)
    worst = 0.0
    for x, y, z in zip(xs, ys, zs):
        bz, by, bx = np.meshgrid((z + off) % L, (y + off) % L, (x + off) % L, indexing="ij")
        block = np.ascontiguousarray(angles_at(before, bx, by, bz))
        cx = block.copy()
        c = np.cos(cx)
        sn = np.sin(cx)
        hx = sum(np.roll(c, sh, ax) for ax in range(3) for sh in (1, -1))[1, 1, 1]
        hy = sum(np.roll(sn, sh, ax) for ax in range(3) for sh in (1, -1))[1, 1, 1]
        oracle.overrelax_half(block, 1)  # local (1, 1, 1) has odd local parity
        d = circ_dist(angles_at(after, x, y, z), block[1, 1, 1])
        h = np.hypot(hx, hy)
        assert d <= OR_A / h + OR_B, (x, y, z, d, h)
        worst = max(worst, d * h)
    # the other colour is untouched
    i = packed_index(xs + 1 - 2 * (xs % 2), ys, zs)  # a colour-1 neighbour in the row
    assert np.array_equal(before[i], after[i])
    del before
    print(f"L=1024: {n} sampled over-relaxation sites, max |d||h| {worst:.2e}")

    # Metropolis half-sweep of colour 1 (pass counter 17): changed sites take
    # their proposal, word 0 (even packed index) or 2 (odd) of the call with
    # counter (p >> 1, 17, 0, slot << 4 | colour << 3 | tag)
    s.metropolis_half(1, 17)
    met = s.get_packed()
    xs, ys, zs = (rng.integers(0, L, 4 * n) for _ in range(3))
    keep = ((xs + ys + zs) % 2) == 1
    xs, ys, zs = xs[keep][:n], ys[keep][:n], zs[keep][:n]
    t0, t1 = angles_at(after, xs, ys, zs), angles_at(met, xs, ys, zs)
    changed = circ_dist(t0, t1) > 0
    key = [SEED & 0xFFFFFFFF, SEED >> 32]
    prop = np.empty(n)
    for k, (x, y, z) in enumerate(zip(xs, ys, zs)):
        p = (int(x) >> 1) + (L // 2) * (int(y) + L * int(z))
        w = oracle.philox4x32_10([p >> 1, 17, 0, (0 << 4) | (1 << 3) | oracle.TAG_MET], key)
        prop[k] = 2 * np.pi * float(int(w[2 if p & 1 else 0]) >> 8) / 2.0 ** 24
    assert np.all(circ_dist(t1[changed], prop[changed]) < 1e-6)
    assert 0.2 < changed.mean() < 0.8
    i = packed_index(xs + 1 - 2 * (xs % 2), ys, zs)  # colour-0 sites unchanged
    assert np.array_equal(after[i], met[i])

    # the fused lattice sums against FP64 sums of the stored vectors, plane by plane
    rec = s.measure()[0]
    E = Mx = My = 0.0
    c0, s0 = plane_vectors(met, 0)
    c, sn = c0, s0
    for z in range(L):
        cn, sn_next = (c0, s0) if z == L - 1 else plane_vectors(met, z + 1)
        Mx += c.sum()
        My += sn.sum()
        E -= (c * np.roll(c, -1, 1) + sn * np.roll(sn, -1, 1)).sum()
        E -= (c * np.roll(c, -1, 0) + sn * np.roll(sn, -1, 0)).sum()
        E -= (c * cn + sn * sn_next).sum()
        c, sn = cn, sn_next
    N = L ** 3
    print(f"L=1024: E {rec['E']:.6f} vs FP64 {E:.6f}; |dE| per bond {abs(rec['E'] - E) / (3 * N):.2e}")
    assert abs(rec["E"] - E) < BOND_TOL * 3 * N
    assert abs(rec["Mx"] - Mx) < SITE_TOL * N and abs(rec["My"] - My) < SITE_TOL * N
