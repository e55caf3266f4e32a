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
