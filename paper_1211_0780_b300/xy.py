"""Python binding of libxy (``include/xy.h``): argument marshalling only.

Every step of the hot path runs in the CUDA library; this module loads the
in-tree ``libxy.so`` with ``ctypes``, allocates the caller-owned device
workspace as a torch uint8 tensor, passes torch's current CUDA stream, and
converts results to numpy.  There is no fallback: if the library or a CUDA
device is missing, the calls raise.
"""

from __future__ import annotations

import ctypes
import json
import os
from typing import Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# The library: libxy.so, or the bounds-checked debug build (libxy_check.so,
# compiled with XY_BOUNDS_CHECK) when XY_LIBRARY names it.
LIB_PATH = os.environ.get("XY_LIBRARY") or os.path.join(_HERE, "libxy.so")
CHECK_LIB_PATH = os.path.join(_HERE, "libxy_check.so")

XY_OK, XY_ERR_ARG, XY_ERR_CUDA, XY_ERR_TIMEOUT, XY_ERR_STATE, XY_ERR_NOMEM, XY_ERR_BOUNDS = 0, -1, -2, -3, -4, -5, -6
EXEC_PLAIN, EXEC_GRAPH, EXEC_PERSISTENT = 0, 1, 2
TAG_INIT, TAG_MET, TAG_PT = 1, 2, 3
TILE_MARCH, TILE_BLOCK, TILE_STREAM, TILE_DIRECT, TILE_ANGLE = 0, 1, 2, 3, 4


class XYError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status} ({strerror(status)})")


class Record(ctypes.Structure):
    """xy_record: the lattice sums of one slot at one measurement."""

    _fields_ = [("E", ctypes.c_double), ("Mx", ctypes.c_double), ("My", ctypes.c_double),
                ("C", ctypes.c_double * 3), ("S", ctypes.c_double * 3), ("beta", ctypes.c_double),
                ("slot", ctypes.c_int32), ("beta_index", ctypes.c_int32), ("sweep", ctypes.c_uint64)]


RECORD_DTYPE = np.dtype([("E", "<f8"), ("Mx", "<f8"), ("My", "<f8"), ("C", "<f8", (3,)),
                         ("S", "<f8", (3,)), ("beta", "<f8"), ("slot", "<i4"),
                         ("beta_index", "<i4"), ("sweep", "<u8")])
assert RECORD_DTYPE.itemsize == ctypes.sizeof(Record) == 96

_lib = None

_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
_U64 = ctypes.c_uint64
_SZ = ctypes.c_size_t
_D = ctypes.c_double

_SIGNATURES = {
    "xy_strerror": (ctypes.c_char_p, [_I]),
    "xy_workspace_bytes": (_SZ, [_I, _P, _P, _I64]),
    "xy_init": (_I, [_P, _I, _P, _P, _P, _U64, _P, _SZ, _I64, _P]),
    "xy_destroy": (_I, [_P]),
    "xy_set_exec": (_I, [_P, _I]),
    "xy_sweep": (_I, [_P, _I, _I, _I, _I, _I]),
    "xy_metropolis_half": (_I, [_P, _I, _U64]),
    "xy_overrelax_half": (_I, [_P, _I]),
    "xy_measure": (_I, [_P, _P]),
    "xy_pt_swap": (_I, [_P, _I, _P]),
    "xy_read_series": (_I, [_P, _P, _I64, _P]),
    "xy_series_count": (_I, [_P, _P]),
    "xy_get_state": (_I, [_P, _P, _P, _P]),
    "xy_set_state": (_I, [_P, _P, _P, _P]),
    "xy_get_accepts": (_I, [_P, _P, _P]),
    "xy_get_packed": (_I, [_P, _P]),
    "xy_set_packed": (_I, [_P, _P]),
    "xy_get_packed_angles": (_I, [_P, _P]),
    "xy_set_packed_angles": (_I, [_P, _P]),
    "xy_host_alloc": (_I, [_SZ, _P]),
    "xy_host_free": (_I, [_P]),
    "xy_debug_draws": (_I, [_P, _I, _I, _I, _U64, _P]),
    "xy_debug_fast_math": (_I, [_I, _I64, _P, _P, _P]),
    "xy_set_tile": (_I, [_P, _I, _I, _I, _I]),
    "xy_get_tile": (_I, [_P, _I, _P, _P, _P]),
    "xy_autotune": (_I, [_P, _I, _I]),
    "xy_device_status": (_I, [_P, _P]),
    "xy_debug_barrier_timeout": (_I, [_P, _I, _P]),
    "xy_debug_stream_timeout": (_I, [_P, _I, _P]),
    "xy_reweight_scratch_bytes": (_SZ, [_I64, _I]),
    "xy_reweight_forward": (_I, [_I64, _P, _P, _P, _P, _P, _D, _I, _P, _I, _P, _P, _P, _P, _SZ, _P]),
    "xy_reweight_backward": (_I, [_I, _P, _I, _P, _P, _P, _P, _P, _P, _P]),
    "xy_reweight_noalloc_capacity_bytes": (_SZ, []),
    "xy_peak_probe": (_I, [_I, _P, _SZ, _P, _P]),
    "xy_reweight_forward_noalloc": (_I, [_I64, _P, _P, _P, _P, _P, _D, _I, _P, _I, _P, _P, _P, _P]),
    "xy_set_betas": (_I, [_P, _I, _P]),
    "xy_ladder_update": (_I, [_I, _P, _P, _D, _P]),
    "xy_multihist_scratch_bytes": (_SZ, [_I64, _I, _I]),
    "xy_multihist_solve": (_I, [_I64, _P, _I, _P, _P, _D, _I, _P, _P, _P, _SZ, _P]),
    "xy_multihist_forward": (_I, [_I64, _P, _P, _P, _P, _P, _I, _P, _P, _P, _I, _P, _I, _P, _P, _P, _P, _SZ, _P]),
    "xy_reweight_bins_scratch_bytes": (_SZ, [_I64, _I, _I]),
    "xy_reweight_bins": (_I, [_I64, _P, _P, _P, _P, _P, _D, _I, _P, _I, _P, _P, _P, _SZ, _P]),
    "xy_fss_resample": (_I, [_I, _I, _P, _I, _P, _P, _P]),
    "xy_fss_curves": (_I, [_I, _I, _P, _I, _P, _P, _P]),
    "xy_fss_crossings": (_I, [_I, _I, _P, _I, _P, _I, _P, _I, _P, _P]),
}


def lib() -> ctypes.CDLL:
    """The loaded library; raises if ``libxy.so`` has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libxy.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(L, name, None)
            if fn is None:
                continue
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def strerror(status: int) -> str:
    try:
        return lib().xy_strerror(int(status)).decode()
    except Exception:  # pragma: no cover - only for messages
        return "?"


def _check(status: int, what: str) -> None:
    if status != XY_OK:
        raise XYError(status, what)


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _require_cuda():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libxy needs a CUDA device; none is available")
    return torch


def _library_id() -> str:
    """Content hash of the loaded libxy.so (a rebuilt library invalidates
    cached tile choices)."""
    import hashlib
    h = hashlib.sha1()
    with open(LIB_PATH, "rb") as f:
        for chunk in iter(lambda: f.read(1 << 20), b""):
            h.update(chunk)
    return h.hexdigest()[:16]


def autotune_cache_key(sim, n_metropolis: int, n_overrelax: int, device: str | None = None,
                       library: str | None = None) -> str:
    """Key of one autotune result: lattice sizes, replicas, pass counts,
    execution mode, device name and library build."""
    if device is None:
        import torch
        device = torch.cuda.get_device_name()
    if library is None:
        library = _library_id()
    return json.dumps({"L": list(sim.L), "R": list(sim.R), "nM": int(n_metropolis), "nOR": int(n_overrelax),
                       "exec": int(getattr(sim, "exec_mode", EXEC_PLAIN)), "device": device,
                       "library": library}, sort_keys=True)


def load_tile_cache(path: str) -> dict:
    """The tile cache at `path` ({key: [[ty, tz, kind], ...]}), empty if the
    file is missing or unreadable."""
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        return {}
    return {k: [tuple(int(x) for x in t) for t in v] for k, v in data.items()} if isinstance(data, dict) else {}


def store_tile_cache(path: str, key: str, tiles) -> None:
    """Adds one result to the tile cache at `path` (written through a
    temporary file and renamed, so readers never see a partial file)."""
    data = {k: [list(t) for t in v] for k, v in load_tile_cache(path).items()}
    data[key] = [list(map(int, t)) for t in tiles]
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


class Simulation:
    """Replicas of periodic L^3 XY lattices on one GPU (one exchange ladder
    per lattice).  Wraps one xy_ctx over a torch-allocated workspace."""

    def __init__(self, L, n_replicas, betas, seed: int = 0x5EED2012,
                 series_capacity: int = 1024, stream=None):
        torch = _require_cuda()
        Ls = [int(L)] if np.isscalar(L) else [int(v) for v in L]
        Rs = [int(n_replicas)] * len(Ls) if np.isscalar(n_replicas) else [int(v) for v in n_replicas]
        b = np.ascontiguousarray(np.asarray(betas, dtype=np.float64).reshape(-1))
        self.L = Ls
        self.R = Rs
        self.n_slots = int(sum(Rs))
        self.betas = b
        self.seed = int(seed)
        self._Ls = np.asarray(Ls, dtype=np.int32)
        self._Rs = np.asarray(Rs, dtype=np.int32)
        lb = lib()
        nbytes = lb.xy_workspace_bytes(len(Ls), _ptr(self._Ls), _ptr(self._Rs), int(series_capacity))
        if nbytes == 0:
            raise XYError(XY_ERR_ARG, "xy_workspace_bytes")
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        # allocated on the context's stream, so that the caching allocator
        # orders any later reuse of the block after that stream's work
        with torch.cuda.stream(stream):
            self.workspace = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
        self._ctx = ctypes.c_void_p()
        _check(lb.xy_init(ctypes.byref(self._ctx), len(Ls), _ptr(self._Ls), _ptr(self._Rs), _ptr(b),
                          self.seed, self.workspace.data_ptr(), int(nbytes), int(series_capacity),
                          int(stream.cuda_stream)), "xy_init")

    # -- lifecycle -----------------------------------------------------
    def close(self) -> None:
        if getattr(self, "_ctx", None) and self._ctx.value:
            lib().xy_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def ctx(self):
        return self._ctx

    # -- the sweep path ------------------------------------------------
    def set_exec(self, mode: int) -> None:
        _check(lib().xy_set_exec(self._ctx, int(mode)), "xy_set_exec")
        self.exec_mode = int(mode)

    def sweep(self, n_metropolis: int, n_overrelax: int, n_sweeps: int = 1,
              measure_every: int = 0, pt_swap_every: int = 0) -> None:
        _check(lib().xy_sweep(self._ctx, int(n_metropolis), int(n_overrelax), int(n_sweeps),
                              int(measure_every), int(pt_swap_every)), "xy_sweep")

    def metropolis_half(self, colour: int, mpass: int) -> None:
        _check(lib().xy_metropolis_half(self._ctx, int(colour), int(mpass)), "xy_metropolis_half")

    def overrelax_half(self, colour: int) -> None:
        _check(lib().xy_overrelax_half(self._ctx, int(colour)), "xy_overrelax_half")

    def measure(self) -> np.ndarray:
        out = np.zeros(self.n_slots, dtype=RECORD_DTYPE)
        _check(lib().xy_measure(self._ctx, _ptr(out)), "xy_measure")
        return out

    def pt_swap(self, parity: int) -> int:
        n = ctypes.c_int(0)
        _check(lib().xy_pt_swap(self._ctx, int(parity), ctypes.byref(n)), "xy_pt_swap")
        return int(n.value)

    def series_count(self) -> int:
        n = ctypes.c_int64(0)
        _check(lib().xy_series_count(self._ctx, ctypes.byref(n)), "xy_series_count")
        return int(n.value)

    def read_series(self) -> np.ndarray:
        n = self.series_count()
        out = np.zeros(max(n, 1), dtype=RECORD_DTYPE)
        got = ctypes.c_int64(0)
        _check(lib().xy_read_series(self._ctx, _ptr(out), len(out), ctypes.byref(got)), "xy_read_series")
        return out[: got.value]

    # -- state ---------------------------------------------------------
    def get_state(self):
        """(angles, perm, counters): angles is a list of (L, L, L) float32
        arrays indexed [z, y, x], one per slot."""
        total = sum(L ** 3 * R for L, R in zip(self.L, self.R))
        flat = np.zeros(total, dtype=np.float32)
        perm = np.zeros(self.n_slots, dtype=np.int32)
        ctr = np.zeros(4, dtype=np.uint64)
        _check(lib().xy_get_state(self._ctx, _ptr(flat), _ptr(perm), _ptr(ctr)), "xy_get_state")
        out, at = [], 0
        for L, R in zip(self.L, self.R):
            for _ in range(R):
                out.append(flat[at:at + L ** 3].reshape(L, L, L))
                at += L ** 3
        return out, perm, ctr

    def set_state(self, angles: Sequence[np.ndarray] | None = None, perm=None, counters=None) -> None:
        a = p = c = None
        if angles is not None:
            a = np.ascontiguousarray(np.concatenate([np.asarray(x, np.float32).reshape(-1) for x in angles]))
        if perm is not None:
            p = np.ascontiguousarray(np.asarray(perm, dtype=np.int32))
        if counters is not None:
            c = np.ascontiguousarray(np.asarray(counters, dtype=np.uint64))
        _check(lib().xy_set_state(self._ctx, _ptr(a) if a is not None else None,
                                  _ptr(p) if p is not None else None,
                                  _ptr(c) if c is not None else None), "xy_set_state")

    def n_packed(self) -> int:
        """Floats of the device state: (cos, sin) of every site of every slot."""
        return int(sum(2 * L ** 3 * R for L, R in zip(self.L, self.R)))

    def get_packed(self, out=None):
        """All spins in the device layout into ``out`` (numpy float32 or a
        pinned CPU torch tensor of n_packed() floats)."""
        if out is None:
            out = np.zeros(self.n_packed(), dtype=np.float32)
        ptr = out.data_ptr() if hasattr(out, "data_ptr") else _ptr(out)
        _check(lib().xy_get_packed(self._ctx, ptr), "xy_get_packed")
        return out

    def set_packed(self, src) -> None:
        buf = src if hasattr(src, "data_ptr") else np.ascontiguousarray(src, dtype=np.float32)
        ptr = buf.data_ptr() if hasattr(buf, "data_ptr") else _ptr(buf)  # buf outlives the call
        _check(lib().xy_set_packed(self._ctx, ptr), "xy_set_packed")

    def n_packed_angles(self) -> int:
        """Floats of the state as angles: every site of every slot."""
        return int(sum(L ** 3 * R for L, R in zip(self.L, self.R)))

    def get_packed_angles(self, out=None):
        """All spins as angles in [0, 2 pi), packed order (per slot: colour 0
        then colour 1), into ``out`` (numpy float32 or a pinned CPU torch
        tensor of n_packed_angles() floats)."""
        if out is None:
            out = np.zeros(self.n_packed_angles(), dtype=np.float32)
        ptr = out.data_ptr() if hasattr(out, "data_ptr") else _ptr(out)
        _check(lib().xy_get_packed_angles(self._ctx, ptr), "xy_get_packed_angles")
        return out

    def set_packed_angles(self, src) -> None:
        """Sets every spin from finite angles in the packed order (converted
        on the device); half the bytes of set_packed."""
        buf = src if hasattr(src, "data_ptr") else np.ascontiguousarray(src, dtype=np.float32)
        ptr = buf.data_ptr() if hasattr(buf, "data_ptr") else _ptr(buf)
        _check(lib().xy_set_packed_angles(self._ctx, ptr), "xy_set_packed_angles")

    def counters(self) -> np.ndarray:
        """{Metropolis passes, sweeps, exchange events, records} (no state copy)."""
        ctr = np.zeros(4, dtype=np.uint64)
        _check(lib().xy_get_state(self._ctx, None, None, _ptr(ctr)), "xy_get_state")
        return ctr

    def set_betas(self, lattice: int, betas) -> None:
        b = np.ascontiguousarray(np.asarray(betas, dtype=np.float64))
        if b.size != self.R[lattice]:
            raise ValueError("one beta per replica of the lattice")
        _check(lib().xy_set_betas(self._ctx, int(lattice), _ptr(b)), "xy_set_betas")
        s0 = sum(self.R[:lattice])
        self.betas = self.betas.copy()
        self.betas[s0:s0 + self.R[lattice]] = b

    def ladder(self, lattice: int) -> np.ndarray:
        """The betas of ladder `lattice` (ascending)."""
        s0 = sum(self.R[:lattice])
        return self.betas[s0:s0 + self.R[lattice]].copy()

    def accepts(self):
        met = np.zeros(self.n_slots, dtype=np.uint64)
        swp = np.zeros(self.n_slots, dtype=np.uint64)
        _check(lib().xy_get_accepts(self._ctx, _ptr(met), _ptr(swp)), "xy_get_accepts")
        return met, swp

    def debug_draws(self, slot: int, colour: int, tag: int, count: int) -> np.ndarray:
        g = 0
        for L, R in zip(self.L, self.R):
            if slot < g + R:
                break
            g += R
        out = np.zeros(L ** 3, dtype=np.uint32)
        _check(lib().xy_debug_draws(self._ctx, int(slot), int(colour), int(tag), int(count), _ptr(out)),
               "xy_debug_draws")
        return out.reshape(-1, 2)

    # -- tuning and diagnostics ----------------------------------------
    def set_tile(self, lattice: int, ty: int, tz: int, kind: int = TILE_BLOCK) -> None:
        _check(lib().xy_set_tile(self._ctx, int(lattice), int(kind), int(ty), int(tz)), "xy_set_tile")

    def get_tile(self, lattice: int):
        """(ty, tz, kind) of one lattice's tile."""
        k, ty, tz = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        _check(lib().xy_get_tile(self._ctx, int(lattice), ctypes.byref(k), ctypes.byref(ty), ctypes.byref(tz)),
               "xy_get_tile")
        return int(ty.value), int(tz.value), int(k.value)

    def autotune(self, n_metropolis: int, n_overrelax: int, cache: str | None = None):
        """Tile search (xy_autotune); returns each lattice's (ty, tz, kind).
        With `cache` (a JSON file path) a previous result for the same
        lattices, replicas, pass counts, execution mode, device and library
        build is applied with xy_set_tile instead of timing again, and a new
        result is stored (see autotune_cache_key)."""
        key = autotune_cache_key(self, n_metropolis, n_overrelax) if cache else None
        if key is not None:
            tiles = load_tile_cache(cache).get(key)
            if tiles is not None and len(tiles) == len(self.L):
                for i, (ty, tz, kind) in enumerate(tiles):
                    self.set_tile(i, ty, tz, kind)
                return [self.get_tile(i) for i in range(len(self.L))]
        _check(lib().xy_autotune(self._ctx, int(n_metropolis), int(n_overrelax)), "xy_autotune")
        tiles = [self.get_tile(i) for i in range(len(self.L))]
        if key is not None:
            store_tile_cache(cache, key, tiles)
        return tiles

    def device_status(self) -> int:
        s = ctypes.c_int(0)
        _check(lib().xy_device_status(self._ctx, ctypes.byref(s)), "xy_device_status")
        return int(s.value)

    def debug_barrier_timeout(self, budget_us: int):
        """Runs the test hook of the persistent launch's bounded waits (every
        block waits for a count nothing raises); returns (status code,
        device status)."""
        s = ctypes.c_int(0)
        rc = lib().xy_debug_barrier_timeout(self._ctx, int(budget_us), ctypes.byref(s))
        return int(rc), int(s.value)

    def debug_stream_timeout(self, budget_us: int):
        """Runs the stream-tile plane-wait test hook (lattice 0 on a stream
        tile); returns (status code, device status)."""
        s = ctypes.c_int(0)
        rc = lib().xy_debug_stream_timeout(self._ctx, int(budget_us), ctypes.byref(s))
        return int(rc), int(s.value)


PEAK_KINDS = {"sfu_sincos": 0, "sfu_ex2": 1, "fp32_fma": 2, "fp64_fma": 3, "int_mul_wide": 4,
              "l2_read_bytes": 5}


class _HostBlock:
    """Owner of one xy_host_alloc block; frees it when collected."""

    def __init__(self, ptr: int):
        self.ptr = ptr

    def __del__(self):
        try:
            lib().xy_host_free(ctypes.c_void_p(self.ptr))
        except Exception:
            pass


def pinned_empty(n: int, dtype=np.float32) -> np.ndarray:
    """A numpy array of n elements in page-locked host memory from
    xy_host_alloc (freed with the array): the host buffer for
    set_packed_angles / get_packed_angles / set_packed / get_packed whose
    copies run at the full host-to-device rate."""
    _require_cuda()
    dt = np.dtype(dtype)
    nbytes = max(int(n), 1) * dt.itemsize
    p = ctypes.c_void_p()
    _check(lib().xy_host_alloc(nbytes, ctypes.byref(p)), "xy_host_alloc")
    raw = (ctypes.c_char * nbytes).from_address(p.value)
    raw._owner = _HostBlock(p.value)  # the array's base keeps the block alive
    return np.frombuffer(raw, dtype=dt, count=int(n))


def peak_probe(kind: str) -> float:
    """Measured operations (or bytes) per second of one unit (see xy_peak_probe)."""
    torch = _require_cuda()
    buf = torch.empty(64 << 20, dtype=torch.uint8, device="cuda")
    out = ctypes.c_double(0.0)
    _check(lib().xy_peak_probe(PEAK_KINDS[kind], buf.data_ptr(), buf.numel(), ctypes.byref(out),
                               torch.cuda.current_stream().cuda_stream), "xy_peak_probe")
    return float(out.value)


def fast_math(kind: str, values) -> np.ndarray:
    """The update's fast-math expressions on the device (see
    xy_debug_fast_math).  kind "proposal": uint32 proposal words -> (n, 2)
    FP32 proposal vectors (cos, sin); kind "accept": FP32 exponents x ->
    the FP32 thresholds exp(x) 2^24; kind "atan2": (n, 2) FP32 pairs
    (x, y) -> the angle-storage tile's atan2(y, x)."""
    torch = _require_cuda()
    k = {"proposal": 0, "accept": 1, "atan2": 2}[kind]
    src = torch.as_tensor(np.ascontiguousarray(values, dtype=np.uint32 if k == 0 else np.float32).view(
        np.int32 if k == 0 else np.float32), device="cuda")
    n = src.numel() // 2 if k == 2 else src.numel()
    out = torch.empty(2 * n if k == 0 else n, dtype=torch.float32, device="cuda")
    _check(lib().xy_debug_fast_math(k, n, src.data_ptr(), out.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream), "xy_debug_fast_math")
    res = out.cpu().numpy()
    return res.reshape(n, 2) if k == 0 else res


# ---------------------------------------------------------------------------
# Single-histogram reweighting (FP64), forward and backward kernels
# ---------------------------------------------------------------------------

OUT_ROWS = ("logZ", "E", "m2", "m4", "csum", "s2sum")
COV_ROWS = ("varE", "m2", "m4", "csum", "s2sum")


def _series_tensors(series, device="cuda"):
    import torch
    E = torch.as_tensor(series["E"], dtype=torch.float64, device=device).contiguous()
    m2 = torch.as_tensor(series["m2"], dtype=torch.float32, device=device).contiguous()
    m4 = torch.as_tensor(series["m4"], dtype=torch.float32, device=device).contiguous()
    c = torch.as_tensor(series["c"], dtype=torch.float32, device=device).contiguous()
    s2 = torch.as_tensor(series["s2"], dtype=torch.float32, device=device).contiguous()
    T = E.numel()
    if m2.numel() != T or m4.numel() != T or c.shape != (3, T) or s2.shape != (3, T):
        raise ValueError("series columns: E[T], m2[T], m4[T], c[3][T], s2[3][T]")
    return E, m2, m4, c, s2


def reweight_forward(series, beta0: float, betap, L: int, scratch=None):
    """Runs the forward kernel.  ``series`` holds E (f64), m2, m4 (f32), c and
    s2 (f32, shape (3, T)), as torch CUDA tensors or arrays.  Returns a dict
    of FP64 CUDA tensors: the rows of OUT_ROWS, U and rhoL, and the
    covariances with E (COV_ROWS, prefixed 'cov_')."""
    import torch
    _require_cuda()
    E, m2, m4, c, s2 = _series_tensors(series)
    bp = torch.as_tensor(betap, dtype=torch.float64, device="cuda").contiguous()
    T, K = E.numel(), bp.numel()
    need = lib().xy_reweight_scratch_bytes(T, K)
    if need == 0:
        raise XYError(XY_ERR_ARG, "xy_reweight_scratch_bytes")
    if scratch is None or scratch.numel() < need:
        scratch = torch.empty(int(need), dtype=torch.uint8, device="cuda")
    out = torch.empty((6, K), dtype=torch.float64, device="cuda")
    obs = torch.empty((3, K), dtype=torch.float64, device="cuda")
    cov = torch.empty((5, K), dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    _check(lib().xy_reweight_forward(T, E.data_ptr(), m2.data_ptr(), m4.data_ptr(), c.data_ptr(),
                                     s2.data_ptr(), float(beta0), K, bp.data_ptr(), int(L),
                                     out.data_ptr(), obs.data_ptr(), cov.data_ptr(),
                                     scratch.data_ptr(), int(scratch.numel()), st), "xy_reweight_forward")
    res = {name: out[i] for i, name in enumerate(OUT_ROWS)}
    res["U"] = obs[0]
    res["rhoL"] = obs[1]
    res["q2"] = obs[2]  # <m^4>/<m^2>^2 (Eq. 11), the ratio of the paper's collapse
    for i, name in enumerate(COV_ROWS):
        res["cov_" + name] = cov[i]
    res["_out"], res["_obs"], res["_cov"] = out, obs, cov
    return res


def reweight_backward(betap, L: int, fwd, gU=None, grhoL=None):
    """Runs the backward kernel: returns (grad_betap or None, dobs[3][K])
    with dobs = {dU/dbeta', d(rho_s L)/dbeta', dq2/dbeta'}."""
    import torch
    bp = torch.as_tensor(betap, dtype=torch.float64, device="cuda").contiguous()
    K = bp.numel()
    dobs = torch.empty((3, K), dtype=torch.float64, device="cuda")
    grad = torch.empty(K, dtype=torch.float64, device="cuda") if (gU is not None or grhoL is not None) else None
    # Keep the contiguous copies alive until the kernel has been enqueued on
    # this stream (the caching allocator then orders any reuse after it).
    gUc = gU.to(torch.float64).contiguous() if gU is not None else None
    gRc = grhoL.to(torch.float64).contiguous() if grhoL is not None else None
    gUp = gUc.data_ptr() if gUc is not None else None
    gRp = gRc.data_ptr() if gRc is not None else None
    st = torch.cuda.current_stream().cuda_stream
    _check(lib().xy_reweight_backward(K, bp.data_ptr(), int(L), fwd["_out"].data_ptr(),
                                      fwd["_cov"].data_ptr(), gUp, gRp,
                                      grad.data_ptr() if grad is not None else None,
                                      dobs.data_ptr(), st), "xy_reweight_backward")
    return grad, dobs


def _make_reweight_fn():
    import torch

    class ReweightFn(torch.autograd.Function):
        """(U_L(beta'), rho_s L(beta')) from a series; differentiable in beta'."""

        @staticmethod
        def forward(ctx, betap, series, beta0, L):
            fwd = reweight_forward(series, beta0, betap.detach(), L)
            ctx.save_for_backward(betap.detach(), fwd["_out"], fwd["_cov"])
            ctx.L = int(L)
            return fwd["U"].clone(), fwd["rhoL"].clone()

        @staticmethod
        def backward(ctx, gU, gR):
            betap, out, cov = ctx.saved_tensors
            gU = gU.to(torch.float64) if gU is not None else torch.zeros_like(betap)
            gR = gR.to(torch.float64) if gR is not None else torch.zeros_like(betap)
            grad, _ = reweight_backward(betap, ctx.L, {"_out": out, "_cov": cov}, gU, gR)
            return grad, None, None, None

    return ReweightFn


_ReweightFn = None


def reweight(series, beta0: float, betap, L: int):
    """Autograd entry point: returns (U_L, rho_s L) at each beta'."""
    global _ReweightFn
    if _ReweightFn is None:
        _ReweightFn = _make_reweight_fn()
    return _ReweightFn.apply(betap, series, float(beta0), int(L))
