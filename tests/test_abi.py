"""The C-ABI library loads on a machine without a GPU, exports every entry
point include/xy.h declares, and rejects invalid arguments on the host
before touching the device (no compute calls here)."""

import ctypes
import os
import re

import numpy as np
import pytest

from paper_1211_0780_b300 import build as xybuild
from paper_1211_0780_b300 import xy

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    xybuild.build()
    return xy.lib()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "xy.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(xy_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(xy._SIGNATURES), set(names) - set(xy._SIGNATURES)


def test_status_strings(lib):
    for code in (0, -1, -2, -3, -4, -5):
        assert xy.strerror(code)
    assert xy.strerror(-1) == "invalid argument"


def _i32(v):
    return np.asarray(v, dtype=np.int32)


def test_workspace_bytes_validation(lib):
    L, R = _i32([16]), _i32([1])
    assert lib.xy_workspace_bytes(1, L.ctypes.data, R.ctypes.data, 10) > 16 ** 3 * 4
    for badL in (12, 4, 0, 2048):
        assert lib.xy_workspace_bytes(1, _i32([badL]).ctypes.data, R.ctypes.data, 10) == 0
    assert lib.xy_workspace_bytes(1, L.ctypes.data, _i32([0]).ctypes.data, 10) == 0
    assert lib.xy_workspace_bytes(0, L.ctypes.data, R.ctypes.data, 10) == 0
    assert lib.xy_workspace_bytes(1, L.ctypes.data, R.ctypes.data, -1) == 0
    # grows with lattices, replicas and the series buffer
    a = lib.xy_workspace_bytes(1, L.ctypes.data, R.ctypes.data, 0)
    b = lib.xy_workspace_bytes(1, L.ctypes.data, _i32([4]).ctypes.data, 0)
    c = lib.xy_workspace_bytes(1, L.ctypes.data, R.ctypes.data, 1000)
    assert b > a and c >= a + 1000 * 96


def test_init_rejects_bad_arguments_before_the_device(lib):
    """Argument checks precede every CUDA call, so these run without a GPU."""
    ctx = ctypes.c_void_p()
    L, R = _i32([16, 24]), _i32([2, 2])
    fake_ws = ctypes.c_void_p(256 * 1024)  # never dereferenced: validation fails first
    good = np.array([0.40, 0.45, 0.40, 0.45])
    cases = [
        (_i32([12, 24]), R, good),                       # L not a multiple of 8
        (L, _i32([2, 0]), good),                         # no replicas
        (L, R, np.array([0.45, 0.40, 0.40, 0.45])),      # not ascending
        (L, R, np.array([0.40, np.nan, 0.40, 0.45])),    # not finite
        (L, R, np.array([-0.1, 0.45, 0.40, 0.45])),      # negative
    ]
    for Ls, Rs, b in cases:
        rc = lib.xy_init(ctypes.byref(ctx), 2, Ls.ctypes.data, Rs.ctypes.data, b.ctypes.data, 1,
                         fake_ws, 1 << 40, 0, None)
        assert rc == xy.XY_ERR_ARG
    # null outputs and misaligned workspace
    assert lib.xy_init(None, 2, L.ctypes.data, R.ctypes.data, good.ctypes.data, 1, fake_ws, 1 << 40, 0, None) == xy.XY_ERR_ARG
    assert lib.xy_init(ctypes.byref(ctx), 2, L.ctypes.data, R.ctypes.data, good.ctypes.data, 1,
                       ctypes.c_void_p(256 * 1024 + 8), 1 << 40, 0, None) == xy.XY_ERR_ARG
    # workspace too small
    assert lib.xy_init(ctypes.byref(ctx), 2, L.ctypes.data, R.ctypes.data, good.ctypes.data, 1,
                       fake_ws, 1024, 0, None) == xy.XY_ERR_NOMEM


def test_null_context_and_reweight_validation(lib):
    assert lib.xy_destroy(None) == 0
    assert lib.xy_sweep(None, 1, 1, 1, 0, 0) == xy.XY_ERR_ARG
    assert lib.xy_set_exec(None, 0) == xy.XY_ERR_ARG
    assert lib.xy_reweight_scratch_bytes(1, 10) == 0
    assert lib.xy_reweight_scratch_bytes(1000, 0) == 0
    n = lib.xy_reweight_scratch_bytes(10 ** 6, 4096)
    assert n >= 4096 * 11 * 8
    p = ctypes.c_void_p(256)
    assert lib.xy_reweight_forward(1, p, p, p, p, p, 0.45, 4, p, 16, p, p, p, p, 1 << 30, None) == xy.XY_ERR_ARG
    assert lib.xy_reweight_forward(1000, p, p, p, p, p, float("nan"), 4, p, 16, p, p, p, p, 1 << 30, None) == xy.XY_ERR_ARG
    assert lib.xy_reweight_forward(1000, p, p, p, p, p, 0.45, 4, p, 16, p, p, p, p, 16, None) == xy.XY_ERR_NOMEM
    assert lib.xy_reweight_backward(0, p, 16, p, p, p, p, p, p, None) == xy.XY_ERR_ARG
    # host buffers: argument errors come back before any CUDA call
    out = ctypes.c_void_p(123)
    assert lib.xy_host_alloc(0, ctypes.byref(out)) == xy.XY_ERR_ARG
    assert lib.xy_host_alloc(16, None) == xy.XY_ERR_ARG
    assert lib.xy_host_free(None) == xy.XY_OK


def test_product_path_has_no_fallback(monkeypatch):
    """Without the built library the binding raises instead of computing."""
    monkeypatch.setattr(xy, "_lib", None)
    monkeypatch.setattr(xy, "LIB_PATH", "/nonexistent/libxy.so")
    with pytest.raises(RuntimeError):
        xy.lib()


def test_scratch_size_queries_on_edge_arguments():
    """The host-side size queries never divide by zero or overflow on edge
    arguments (0 = invalid)."""
    from paper_1211_0780_b300 import xy
    lb = xy.lib()
    assert lb.xy_multihist_scratch_bytes(1000, 4, 0) > 0
    assert lb.xy_multihist_scratch_bytes(1000, 4, 1) > 0
    assert lb.xy_multihist_scratch_bytes(1000, 257, 4) == 0
    assert lb.xy_multihist_scratch_bytes(0, 4, 4) == 0
    assert lb.xy_reweight_bins_scratch_bytes(1000, 1, 1000) > 0
    assert lb.xy_reweight_bins_scratch_bytes(1000, 1, 1001) == 0
    assert lb.xy_reweight_scratch_bytes(2, 1) > 0 and lb.xy_reweight_scratch_bytes(1, 1) == 0
