"""Multi-histogram reweighting of a whole parallel-tempering ladder
(Ferrenberg and Swendsen, 1989): the records of all R couplings pooled,
free energies solved self-consistently on the device, and averages (with
covariances for beta' derivatives) at any target couplings.

Marshalling only: ``xy_multihist_solve`` / ``xy_multihist_forward`` do the
work.  A series here is the dict of the single-histogram functions (E f64,
m2, m4 f32, c, s2 f32 of shape (3, T)) with the records of all couplings
pooled; ``betas`` and ``counts`` say how many records each coupling gave.
"""

from __future__ import annotations

import numpy as np

import ctypes

from . import xy


def pool(series_list):
    """Concatenates per-coupling series into one pooled series; returns
    (pooled, counts)."""
    out = {"E": np.concatenate([np.asarray(s["E"], np.float64) for s in series_list]),
           "m2": np.concatenate([np.asarray(s["m2"], np.float32) for s in series_list]),
           "m4": np.concatenate([np.asarray(s["m4"], np.float32) for s in series_list]),
           "c": np.concatenate([np.asarray(s["c"], np.float32) for s in series_list], axis=1),
           "s2": np.concatenate([np.asarray(s["s2"], np.float32) for s in series_list], axis=1)}
    counts = np.array([len(s["E"]) for s in series_list], dtype=np.int64)
    return out, counts


def series_from_records(rec, L: int, n_ladder: int):
    """Splits a read_series() record array of one ladder by beta index:
    returns (list of per-coupling series, betas)."""
    N = float(L) ** 3
    out, betas = [], []
    for k in range(n_ladder):
        r = rec[rec["beta_index"] == k]
        m2 = (r["Mx"] ** 2 + r["My"] ** 2) / N ** 2
        out.append({"E": r["E"].astype(np.float64), "m2": m2.astype(np.float32), "m4": (m2 * m2).astype(np.float32),
                    "c": (r["C"].T / N).astype(np.float32), "s2": (r["S"].T ** 2 / N).astype(np.float32)})
        betas.append(float(r["beta"][0]))
    return out, np.asarray(betas)


def solve(pooled, betas, counts, tol: float = 1e-10, max_iter: int = 10000, f0=None, scratch=None):
    """Free energies f[R] (f_0 = 0) and the iteration count."""
    import torch
    E = torch.as_tensor(pooled["E"], dtype=torch.float64, device="cuda").contiguous()
    b = np.ascontiguousarray(betas, dtype=np.float64)
    n = np.ascontiguousarray(counts, dtype=np.int64)
    R, T = b.size, E.numel()
    need = xy.lib().xy_multihist_scratch_bytes(T, R, 0)
    if need == 0:
        raise xy.XYError(xy.XY_ERR_ARG, "xy_multihist_scratch_bytes")
    if scratch is None or scratch.numel() < need:
        scratch = torch.empty(int(need), dtype=torch.uint8, device="cuda")
    f = np.zeros(R) if f0 is None else np.ascontiguousarray(f0, dtype=np.float64).copy()
    it = ctypes.c_int(0)
    xy._check(xy.lib().xy_multihist_solve(T, E.data_ptr(), R, xy._ptr(b), xy._ptr(n), float(tol), int(max_iter),
                                          xy._ptr(f), ctypes.byref(it), scratch.data_ptr(), int(scratch.numel()),
                                          torch.cuda.current_stream().cuda_stream), "xy_multihist_solve")
    return f, int(it.value)


def forward(pooled, betas, counts, f, betap, L: int, scratch=None):
    """Averages at each beta' (dict like xy.reweight_forward's)."""
    import torch
    E, m2, m4, c, s2 = xy._series_tensors(pooled)
    bp = torch.as_tensor(betap, dtype=torch.float64, device="cuda").contiguous()
    b = np.ascontiguousarray(betas, dtype=np.float64)
    n = np.ascontiguousarray(counts, dtype=np.int64)
    fv = np.ascontiguousarray(f, dtype=np.float64)
    T, K, R = E.numel(), bp.numel(), b.size
    need = xy.lib().xy_multihist_scratch_bytes(T, R, K)
    if need == 0:
        raise xy.XYError(xy.XY_ERR_ARG, "xy_multihist_scratch_bytes")
    if scratch is None or scratch.numel() < need:
        scratch = torch.empty(int(need), dtype=torch.uint8, device="cuda")
    out = torch.empty((6, K), dtype=torch.float64, device="cuda")
    obs = torch.empty((3, K), dtype=torch.float64, device="cuda")
    cov = torch.empty((5, K), dtype=torch.float64, device="cuda")
    xy._check(xy.lib().xy_multihist_forward(T, E.data_ptr(), m2.data_ptr(), m4.data_ptr(), c.data_ptr(),
                                            s2.data_ptr(), R, xy._ptr(b), xy._ptr(n), xy._ptr(fv), K, bp.data_ptr(),
                                            int(L), out.data_ptr(), obs.data_ptr(), cov.data_ptr(),
                                            scratch.data_ptr(), int(scratch.numel()),
                                            torch.cuda.current_stream().cuda_stream), "xy_multihist_forward")
    res = {name: out[i] for i, name in enumerate(xy.OUT_ROWS)}
    res["U"], res["rhoL"], res["q2"] = obs[0], obs[1], obs[2]
    for i, name in enumerate(xy.COV_ROWS):
        res["cov_" + name] = cov[i]
    res["_out"], res["_obs"], res["_cov"] = out, obs, cov
    return res
