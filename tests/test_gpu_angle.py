"""The angle-storage tile kind (kind 4): a lattice kept as FP32 angles (4
bytes per spin) instead of vectors, for states larger than L2.

Against the oracle on the stored angles themselves (they convert to FP64
exactly): Metropolis half-sweeps within 1e-5 rad outside accept margins
below 1e-6 (counted), over-relaxation half-sweeps within the conditioning
bound below at every site and 99.9% of the sites within 1e-5 rad, the
lattice sums, a whole sweep equal to its half-sweeps issued one by one, and
the same spins bit for bit in every execution mode and tile shape of the
kind.  Changing the kind converts the stored state in place.
"""

import numpy as np
import pytest

import oracle
from helpers import circ_dist, stored_angles64

pytestmark = pytest.mark.gpu

SEED = 0x5EED2012
ANGLE = 4
TOL_RAD, MARGIN = 1e-5, 1e-6
# Over-relaxation (Eq. 2) on stored angles, theta' = 2 phi - theta with phi
# the field's angle: every neighbour's vector comes from the fast sincos
# (<= 3.5e-7 per component, measured <= 3.4e-7; as a vector error <= 4.3e-7
# with the measured length error), six of them and the FP32 field sum
# (<= 1.2e-6 per component) move the field by <= 3.8e-6 and phi by
# <= |dh| / |h|, which the reflection doubles; the tile's atan2 (<= 4e-7,
# test_gpu_accuracy; the bound keeps atan2f's 3 ulp, 7.2e-7, doubled), the
# one rounding of 2 phi - theta (<= 4.8e-7, |2 phi - theta| < 4 pi) and up
# to two additions of the FP32 2 pi to take it into [0, 2 pi)
# (<= 1.75e-7 + 2.4e-7 each) add a constant.
OR_A, OR_B = 7.6e-6, 2.8e-6
BOND_TOL, SITE_TOL = 2e-6, 1e-6


def sim(L, R, betas, seed=SEED, **kw):
    from paper_1211_0780_b300 import xy
    return xy.Simulation(L, R, betas, seed, **kw)


def field_norm(theta):
    c, s = np.cos(theta), np.sin(theta)
    hx = sum(np.roll(c, sh, ax) for ax in range(3) for sh in (1, -1))
    hy = sum(np.roll(s, sh, ax) for ax in range(3) for sh in (1, -1))
    return np.hypot(hx, hy)


def colour_mask(L, colour):
    z, y, x = np.meshgrid(*(np.arange(L),) * 3, indexing="ij")
    return ((x + y + z) % 2) == colour


TILES = [(16, (16, 16)), (24, (5, 7)), (40, (8, 40)), (40, (3, 16)), (8, (1, 8))]


@pytest.mark.parametrize("L,tile", TILES)
def test_angle_half_sweeps_against_oracle(L, tile):
    beta = 0.4542
    s = sim(L, 1, [beta])
    s.set_tile(0, *tile, ANGLE)
    s.sweep(1, 1, 3)
    pk = s.get_packed()
    th = stored_angles64(s, pk)[0]
    assert th.min() >= 0.0 and th.max() < 2 * np.pi
    excluded = 0
    for colour, mpass in ((0, 3), (1, 9)):
        s.set_packed(pk)
        s.metropolis_half(colour, mpass)
        g = stored_angles64(s)[0]
        ref = th.copy()
        _, margin = oracle.metropolis_half(ref, beta, SEED, 0, mpass, colour, want_margin=True)
        close = margin < MARGIN
        excluded += int(close.sum())
        assert np.max(circ_dist(g, ref)[~close]) < TOL_RAD
        assert np.all(g[~colour_mask(L, colour)] == th[~colour_mask(L, colour)])
    assert excluded <= max(2, 1e-4 * L ** 3)
    for colour in (0, 1):
        s.set_packed(pk)
        s.overrelax_half(colour)
        g = stored_angles64(s)[0]
        ref = th.copy()
        h = field_norm(ref)
        oracle.overrelax_half(ref, colour)
        m = colour_mask(L, colour)
        d = circ_dist(g, ref)
        print(f"angle storage L={L} tile={tile} colour={colour}: 0.999-quantile {np.quantile(d[m], 0.999):.2e} "
              f"rad, max |d||h| {np.max(d[m] * h[m]):.2e}")
        assert np.all(d[m] <= OR_A / h[m] + OR_B), float(np.max(d[m] * h[m]))
        assert np.quantile(d[m], 0.999) < TOL_RAD
        assert np.all(d[~m] == 0)
        assert g.min() >= 0.0 and g.max() < 2 * np.pi


def test_angle_sweep_equals_its_half_sweeps_and_measures():
    """xy_sweep on the angle kind equals the same half-sweeps issued one by
    one, bit for bit, and the fused lattice sums agree with the oracle's
    sums of the stored angles (each term's vectors from the fast sincos:
    <= 2e-6 per bond, <= 1e-6 per site)."""
    L, beta = 24, 0.4542
    a, b = sim(L, 2, [0.44, beta]), sim(L, 2, [0.44, beta])
    for x in (a, b):
        x.set_tile(0, 6, 8, ANGLE)
    a.sweep(1, 2, 1)
    for c in (0, 1):
        b.metropolis_half(c, 0)
    for _ in range(2):
        for c in (0, 1):
            b.overrelax_half(c)
    assert np.array_equal(a.get_packed(), b.get_packed())
    rec = a.measure()
    N = L ** 3
    for slot, th in enumerate(stored_angles64(a)):
        ref = oracle.measure(th)
        assert abs(rec["E"][slot] - ref.E) < BOND_TOL * 3 * N
        assert abs(rec["Mx"][slot] - ref.Mx) < SITE_TOL * N
        assert np.max(np.abs(rec["C"][slot] - ref.C)) < BOND_TOL * N
        assert np.max(np.abs(rec["S"][slot] - ref.S)) < BOND_TOL * N


def test_angle_exec_modes_and_tile_shapes_bit_identical():
    """Plain launches, the CUDA graph and the persistent launches give the
    same angles, permutations and records on the angle kind; so do other
    tile shapes of the kind."""
    from paper_1211_0780_b300 import xy
    Ls, Rs = [16, 24], [3, 2]
    betas = [0.40, 0.45, 0.48, 0.44, 0.46]
    outs = []
    for mode in (xy.EXEC_PLAIN, xy.EXEC_GRAPH, xy.EXEC_PERSISTENT):
        s = sim(Ls, Rs, betas, series_capacity=32)
        s.set_tile(0, 4, 8, ANGLE)
        s.set_tile(1, 6, 4, ANGLE)
        s.set_exec(mode)
        s.sweep(1, 2, 6, measure_every=2, pt_swap_every=1)
        outs.append((s.get_packed(), s.get_state()[1], s.read_series()))
    for other in outs[1:]:
        assert np.array_equal(outs[0][0], other[0])
        assert np.array_equal(outs[0][1], other[1])
        assert outs[0][2].tobytes() == other[2].tobytes()
    res = []
    for tile in ((8, 8), (5, 3), (40, 2), (1, 40)):
        s = sim(40, 1, [0.4542])
        s.set_tile(0, *tile, ANGLE)
        s.sweep(1, 3, 3)
        res.append(s.get_packed())
    assert all(np.array_equal(res[0], r) for r in res[1:])


def test_storage_conversion_keeps_the_state():
    """Changing a lattice between a vector kind and the angle kind converts
    its state in place: the angles read back agree within the conversion's
    rounding (atan2f and sincosf, <= 1e-6 rad), and the kind's own state
    interface (get_state, set_state, set_packed_angles, get_packed_angles)
    reads and writes angles."""
    from paper_1211_0780_b300.inputs import random_angles
    L = 24
    s = sim(L, 2, [0.44, 0.45])
    s.sweep(1, 2, 2)
    before = s.get_state()[0]
    s.set_tile(0, 6, 8, ANGLE)
    mid = s.get_state()[0]
    assert all(np.max(circ_dist(x, y)) < 1e-6 for x, y in zip(before, mid))
    s.set_tile(0, 6, 8, 3)
    after = s.get_state()[0]
    assert all(np.max(circ_dist(x, y)) < 2e-6 for x, y in zip(before, after))
    # the angle kind's state interface: exact round trips of the angles
    s.set_tile(0, 6, 8, ANGLE)
    st = [random_angles((L, L, L), 5 + r).astype(np.float32) for r in range(2)]
    s.set_state(st)
    got = s.get_state()[0]
    assert all(np.max(circ_dist(x, y)) < 1e-7 for x, y in zip(got, st))
    packed = s.get_packed_angles()
    s.set_packed_angles(packed)
    assert np.array_equal(s.get_packed_angles(), packed)
    # angles outside [0, 2 pi) are taken into it
    s.set_state([st[0] + np.float32(2 * np.pi), st[1] - np.float32(2 * np.pi)])
    got = s.get_state()[0]
    assert all(np.max(circ_dist(x, y)) < 1e-6 for x, y in zip(got, st))
    assert all(x.min() >= 0 and x.max() < 2 * np.pi for x in got)


def test_angle_checkpoint_resume_is_bit_exact():
    L = 32
    a = sim(L, 1, [0.4542], series_capacity=8)
    a.set_tile(0, 8, 8, ANGLE)
    a.sweep(1, 3, 4)
    pk, (_, perm, ctr) = a.get_packed(), a.get_state()
    a.sweep(1, 3, 5, measure_every=5)
    b = sim(L, 1, [0.4542], series_capacity=8)
    b.set_tile(0, 8, 8, ANGLE)
    b.set_packed(pk)
    b.set_state(None, perm, ctr)
    b.sweep(1, 3, 5, measure_every=5)
    assert np.array_equal(a.get_packed(), b.get_packed())
    assert a.read_series().tobytes() == b.read_series().tobytes()
