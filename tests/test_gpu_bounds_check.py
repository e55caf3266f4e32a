"""The bounds-checked debug build (libxy_check.so, XY_BOUNDS_CHECK): over
every tile kind, lattice size class, execution mode, the measurement (every
sum, or the energy alone on sweeps that only exchange) and the exchange, no
spin access falls outside its slot (the status word stays 0, so
no XY_ERR_BOUNDS) and the spins and records equal the release library's, bit
for bit.  This is the project's stand-in for compute-sanitizer's memcheck on
the sweep kernels."""

import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys
import numpy as np
from paper_1211_0780_b300 import xy
out = {}
# (lattice sizes, replicas, tile per lattice); tiles ragged in y and z
cases = [([16], [2], [(4, 8, 0)]), ([24], [1], [(5, 7, 1)]), ([40], [1], [(3, 16, 2)]),
         ([24], [2], [(5, 7, 3)]), ([64], [2], [(8, 8, 3)]), ([8], [1], [(1, 8, 3)]),
         ([40], [1], [(40, 2, 3)]), ([80], [1], [(6, 9, 3)]), ([16, 24], [3, 2], [(4, 8, 3), (3, 5, 3)]),
         ([16, 24], [3, 2], [(4, 8, 0), (3, 5, 0)]), ([24], [2], [(5, 7, 4)]), ([40], [1], [(40, 2, 4)]),
         ([16, 24], [3, 2], [(4, 8, 4), (3, 5, 4)])]
for i, (Ls, Rs, tiles) in enumerate(cases):
    for mode in (xy.EXEC_PLAIN, xy.EXEC_GRAPH, xy.EXEC_PERSISTENT):
        if mode == xy.EXEC_PERSISTENT and any(t[2] == 2 for t in tiles):
            continue
        betas = np.concatenate([np.linspace(0.44, 0.46, R) for R in Rs])
        s = xy.Simulation(Ls, Rs, betas, 11 + i, series_capacity=16)
        for j, t in enumerate(tiles):
            s.set_tile(j, *t)
        s.set_exec(mode)
        s.sweep(1, 2, 3, measure_every=1, pt_swap_every=1)
        s.sweep(2, 0, 1, measure_every=1, pt_swap_every=1)
        # exchanges without records: the energy-only measuring kernels
        s.sweep(1, 2, 2, measure_every=0, pt_swap_every=1)
        s.sweep(2, 0, 1, measure_every=0, pt_swap_every=1)
        assert s.device_status() == 0, (i, mode)
        out[f"{i}-{mode}-p"] = s.get_packed()
        out[f"{i}-{mode}-r"] = s.read_series()
np.savez(sys.argv[1], **out)
"""


def run(path, library=None):
    env = dict(os.environ)
    env.pop("XY_LIBRARY", None)
    if library:
        env["XY_LIBRARY"] = library
    subprocess.run([sys.executable, "-c", SCRIPT, path], env=env, check=True, timeout=900, cwd=ROOT)
    return np.load(path)


def test_bounds_checked_build_matches_release(tmp_path):
    from paper_1211_0780_b300 import xy
    assert os.path.exists(xy.CHECK_LIB_PATH), "libxy_check.so not built"
    rel = run(str(tmp_path / "release.npz"))
    chk = run(str(tmp_path / "checked.npz"), xy.CHECK_LIB_PATH)
    assert sorted(rel.files) == sorted(chk.files) and len(rel.files) >= 50
    for k in rel.files:
        assert np.array_equal(rel[k], chk[k]), k
