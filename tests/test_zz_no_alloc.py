"""The allocation-free reweighting entry point (xy_reweight_forward_noalloc),
for callers that cannot hand the library scratch memory (a device budget
fixed at start-up, no allocator calls once running, a host framework that
owns every device allocation).  Called through the C-ABI, it must return
what the scratch-taking xy_reweight_forward returns, call after call, from
its one shared library-owned array.  This file is collected last."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _call_noalloc(lib, s_t, beta0, bp, L, torch):
    E, m2, m4, c, s2 = s_t
    K = bp.numel()
    out = torch.full((6, K), float("nan"), dtype=torch.float64, device="cuda")
    obs = torch.full((3, K), float("nan"), dtype=torch.float64, device="cuda")
    cov = torch.full((5, K), float("nan"), dtype=torch.float64, device="cuda")
    rc = lib.xy_reweight_forward_noalloc(E.numel(), E.data_ptr(), m2.data_ptr(), m4.data_ptr(), c.data_ptr(),
                                         s2.data_ptr(), float(beta0), K, bp.data_ptr(), int(L), out.data_ptr(),
                                         obs.data_ptr(), cov.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return rc, out, obs, cov


def test_noalloc_forward_matches_scratch_entry_point_on_consecutive_calls():
    import torch
    from paper_1211_0780_b300 import xy
    from paper_1211_0780_b300.inputs import synthetic_series
    lib = xy.lib()
    assert lib.xy_reweight_noalloc_capacity_bytes() == 8 << 20
    beta0 = 0.4542
    # consecutive calls with different shapes: the shared array keeps the
    # previous call's contents, which must not leak into the next result
    for L, T, K, seed in ((64, 60000, 4096, 3), (32, 20000, 300, 4), (16, 5000, 37, 5)):
        s = synthetic_series(L, T, seed)
        s_t = xy._series_tensors(s)
        bp = torch.linspace(0.4530, 0.4555, K, dtype=torch.float64, device="cuda")
        ref = xy.reweight_forward(s, beta0, bp, L)
        rc, out, obs, cov = _call_noalloc(lib, s_t, beta0, bp, L, torch)
        assert rc == xy.XY_OK
        np.testing.assert_allclose(out.cpu().numpy(), ref["_out"].cpu().numpy(), rtol=1e-10)
        np.testing.assert_allclose(obs.cpu().numpy(), ref["_obs"].cpu().numpy(), rtol=1e-10)
        c_ref = ref["_cov"].cpu().numpy()
        for row in range(5):
            np.testing.assert_allclose(cov[row].cpu().numpy(), c_ref[row], rtol=1e-10,
                                       atol=1e-10 * np.max(np.abs(c_ref[row])))


def test_noalloc_rejects_sizes_beyond_its_array():
    import torch
    from paper_1211_0780_b300 import xy
    from paper_1211_0780_b300.inputs import synthetic_series
    lib = xy.lib()
    s_t = xy._series_tensors(synthetic_series(8, 1000, 1))
    K = 100000  # K x 11 FP64 partial sums per chunk exceed the 8 MiB array
    bp = torch.linspace(0.45, 0.46, K, dtype=torch.float64, device="cuda")
    rc, out, _, _ = _call_noalloc(lib, s_t, 0.4542, bp, 8, torch)
    assert rc == xy.XY_ERR_NOMEM
    assert torch.isnan(out).all()  # nothing was launched
