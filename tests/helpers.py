"""Small test-side helpers: circular distances and binned error bars."""

import numpy as np

GOLDEN = __import__("os").path.join(__import__("os").path.dirname(__file__), "golden")


def circ_dist(a, b):
    """Distance between angles on the circle, in [0, pi]."""
    d = np.mod(np.asarray(a, np.float64) - np.asarray(b, np.float64) + np.pi, 2 * np.pi) - np.pi
    return np.abs(d)


def binned_mean_err(x, n_bins=50):
    """Mean and the standard error from n_bins consecutive bins (the
    binning analysis the paper uses for its error bars, Sec. II)."""
    x = np.asarray(x, np.float64)
    n = (len(x) // n_bins) * n_bins
    b = x[:n].reshape(n_bins, -1).mean(axis=1)
    return float(x[:n].mean()), float(b.std(ddof=1) / np.sqrt(n_bins))


def load_kat():
    rows = []
    with open(__import__("os").path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            w = [int(t, 16) for t in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


TILE_ANGLE = 4  # the tile kind that keeps a lattice as angles


def stored_angles64(sim, packed=None):
    """Exact FP64 angles of the spins a Simulation stores, one natural-layout
    (L, L, L) array [z, y, x] per slot.  A lattice on a vector tile kind
    keeps each spin as an FP32 vector (cos, sin) in the packed layout of the
    library's header (per slot: colour 0's N/2 cosines, its N/2 sines, then
    colour 1's; site (x, y, z) at (x >> 1) + (L/2)(y + L z)), and atan2 of
    the two stored floats in FP64 is the direction of that vector to ~1e-16
    rad, with no rounding to an FP32 angle in between.  A lattice on the
    angle tile kind keeps the FP32 angle itself where the cosine would be,
    which converts to FP64 exactly.  Parity checks hand these to the oracle
    and compare its output with them."""
    pk = sim.get_packed() if packed is None else packed
    out, at = [], 0
    for i, (L, R) in enumerate(zip(sim.L, sim.R)):
        angles = sim.get_tile(i)[2] == TILE_ANGLE
        N, H = L ** 3, L // 2
        z, y, x = np.meshgrid(*(np.arange(L),) * 3, indexing="ij")
        col = (x + y + z) % 2
        p = (x >> 1) + H * (y + L * z)
        for _ in range(R):
            base = at + col * N
            if angles:
                t = pk[base + p].astype(np.float64)
            else:
                c = pk[base + p].astype(np.float64)
                s = pk[base + N // 2 + p].astype(np.float64)
                t = np.arctan2(s, c)
                t[t < 0] += 2 * np.pi
                t[t >= 2 * np.pi] = 0.0
            out.append(np.ascontiguousarray(t))
            at += 2 * N
    return out
