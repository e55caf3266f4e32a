#!/usr/bin/env python3
"""Throughput of the 3D XY sweep path on B300: spin updates per ns.

Headline workload (one GPU): a 160^3 periodic lattice, one replica,
beta = 0.4542, sweeps of 1 Metropolis + 5 over-relaxation passes, the
lattice sums measured every 10 sweeps.  One step = 10 sweeps + the fused
measurement = 10 * 6 * 160^3 = 245,760,000 spin updates.  The lattice
(16.4 MB) is smaller than L2, so L2 is flushed (a 256 MB write) before every
timed step, outside its CUDA-event bracket.

Also reported (extra keys): the batched parallel-tempering workload (64^3 x
32 replicas, 1 + 3 passes, exchange every sweep) batched into each
half-sweep kernel (CUDA graph) and in the persistent launches vs the plain
per-replica launch loop, the ragged batch,
and reweighting throughput.

--impl reference runs the FP64 CPU oracle (the reference arm of this build)
on the host cores, on bounded samples of the same workload.

Under torchrun every rank runs an independent replica (the path has no
exchange between GPUs); rank 0 prints one JSON line.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

SEED = 0x5EED2012
L_MAIN, BETA_MAIN, NM_MAIN, NOR_MAIN, SWEEPS_PER_STEP = 160, 0.4542, 1, 5, 10
UPDATES_PER_STEP = SWEEPS_PER_STEP * (NM_MAIN + NOR_MAIN) * L_MAIN ** 3
METRIC = "XY spin updates/ns at L=160, plain vs batched PT; % of HBM/SFU roofline"
UNIT = "spin updates/ns"
WORKLOAD = ("160^3 periodic XY lattice, 1 replica, beta=0.4542, sweep = 1 Metropolis + 5 "
            "over-relaxation passes, lattice sums every 10 sweeps; step = 10 sweeps")
# Algorithmic bytes of one site update: read own angle 4 B, write it 4 B,
# read the other colour once 4 B (halo re-reads excluded).
BYTES_PER_UPDATE = 12


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6400.0)), "measured"
    return 6400.0, "fallback"


class ClockSampler:
    """SM clocks and throttle reasons sampled during the timed region: NVML
    polled every 2 ms from a background thread (the timed region of a short
    run lasts milliseconds), else nvidia-smi at its 200 ms minimum."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None
        self.thread = None
        self.samples = []
        self.source = None

    # NVML (nvml.h): NVML_CLOCK_SM and the clock-event reason bits
    NVML_CLOCK_SM = 1
    BITS = (("hw_slowdown", 0x8), ("hw_thermal_slowdown", 0x40), ("sw_thermal_slowdown", 0x20),
            ("sw_power_cap", 0x4))

    def _nvml_loop(self, lib, handle, reasons_fn):
        import ctypes
        sm, mx, mask = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        while not self.stop_flag.is_set():
            if (lib.nvmlDeviceGetClockInfo(handle, self.NVML_CLOCK_SM, ctypes.byref(sm)) != 0
                    or lib.nvmlDeviceGetMaxClockInfo(handle, self.NVML_CLOCK_SM, ctypes.byref(mx)) != 0
                    or reasons_fn(handle, ctypes.byref(mask)) != 0):
                break
            self.samples.append((float(sm.value), float(mx.value), [n for n, bit in self.BITS if mask.value & bit]))
            time.sleep(0.001)

    def start(self):
        try:
            import ctypes
            import threading
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            handle = ctypes.c_void_p()
            if lib.nvmlInit_v2() != 0 or lib.nvmlDeviceGetHandleByIndex_v2(self.index, ctypes.byref(handle)) != 0:
                raise OSError("nvml")
            reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                lib.nvmlDeviceGetCurrentClocksThrottleReasons
            # one query of each kind before the timed region (not recorded):
            # the first calls are slow, and the region is only milliseconds
            v, m = ctypes.c_uint(), ctypes.c_ulonglong()
            lib.nvmlDeviceGetClockInfo(handle, self.NVML_CLOCK_SM, ctypes.byref(v))
            lib.nvmlDeviceGetMaxClockInfo(handle, self.NVML_CLOCK_SM, ctypes.byref(v))
            reasons_fn(handle, ctypes.byref(m))
            self.stop_flag = threading.Event()
            self.thread = threading.Thread(target=self._nvml_loop, args=(lib, handle, reasons_fn), daemon=True)
            self.thread.start()
            self.source = "nvml, 1 ms"
            return
        except (OSError, AttributeError):
            self.thread = None
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            self.source = "nvidia-smi, 200 ms"
        except OSError:
            self.proc = None

    def stop(self):
        sm, mx, reasons = [], [], set()
        if self.thread is not None:
            self.stop_flag.set()
            self.thread.join(timeout=5)
            for a, b, r in self.samples:
                sm.append(a)
                mx.append(b)
                reasons.update(r)
        elif self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            with open(self.path) as f:
                for line in f:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) < 9:
                        continue
                    try:
                        sm.append(float(parts[1]))
                        mx.append(float(parts[2]))
                    except ValueError:
                        continue
                    for name, v in zip(self.NAMES, parts[5:9]):
                        if v.lower() == "active":
                            reasons.add(name)
            os.unlink(self.path)
        else:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no clock source"], "samples": 0}
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm), "source": self.source}


def allreduce_max(value: float, world: int) -> float:
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------- CPU oracle

def workload_config(world: int) -> dict:
    """The headline workload as both arms run it (the `config` of the line)."""
    return {"workload": WORKLOAD, "L": L_MAIN, "replicas": 1, "beta": BETA_MAIN,
            "sweeps_per_step": SWEEPS_PER_STEP, "measure_every": SWEEPS_PER_STEP,
            "updates_per_step": UPDATES_PER_STEP,
            "l2": "GPU arm: flushed (256 MB write) before every timed step",
            "parallelism": f"replicas only x{world}"}


def oracle_step(th, mpass: int) -> int:
    """One step of the headline workload on the FP64 oracle: SWEEPS_PER_STEP
    sweeps of 1 + 5 passes with the lattice sums after the last one.
    Returns the next Metropolis-pass counter."""
    import oracle
    oracle.run_chain(th, BETA_MAIN, SEED, 0, mpass, NM_MAIN, NOR_MAIN, SWEEPS_PER_STEP, SWEEPS_PER_STEP)
    return mpass + SWEEPS_PER_STEP * NM_MAIN


def oracle_rate(seconds: float, threads: int | None = None, sweeps: int = SWEEPS_PER_STEP):
    """FP64 oracle on the host cores: steps of the headline workload (or,
    with sweeps=1, single unmeasured sweeps) until about `seconds` have
    passed.  Returns (updates/ns, threads, sweeps done)."""
    import oracle
    n = threads or os.cpu_count() or 1
    oracle.set_threads(n)
    th = oracle.init_uniform((L_MAIN,) * 3, SEED, 0)
    done, elapsed = 0, 0.0
    mpass = 0
    while elapsed < seconds or done == 0:
        t0 = time.perf_counter()
        if sweeps == SWEEPS_PER_STEP:
            mpass = oracle_step(th, mpass)
        else:
            oracle.run_chain(th, BETA_MAIN, SEED, 0, mpass, NM_MAIN, NOR_MAIN, sweeps, 0)
            mpass += sweeps * NM_MAIN
        elapsed += time.perf_counter() - t0
        done += sweeps
    upd = done * (NM_MAIN + NOR_MAIN) * L_MAIN ** 3
    return upd / (elapsed * 1e9), n, done


def cpu_model() -> str:
    """The host CPU's model name (Linux /proc/cpuinfo), or "unknown"."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    n = os.cpu_count() or 1
    oracle.set_threads(n)
    th = oracle.init_uniform((L_MAIN,) * 3, SEED, 0)
    mpass = 0
    for _ in range(args.warmup):
        mpass = oracle_step(th, mpass)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        mpass = oracle_step(th, mpass)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = args.steps * UPDATES_PER_STEP / (total * 1e9)
    sample = (f"{args.steps} steps of {SWEEPS_PER_STEP} sweeps (1 Metropolis + 5 over-relaxation passes) of the "
              f"160^3 lattice with the lattice sums after each step's last sweep: the workload's own steps")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "device": f"host CPU ({cpu_model()}), {n} threads (the FP64 oracle; rank 0 only)",
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(world),
        "exec": "FP64 oracle in C, OpenMP over the sites of each half-sweep",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": n, "kind": "oracle", "sample": sample,
                         "cpu_model": cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- GPU arm

def time_kernel(fn, stream, n, warm=5):
    """Average device time of one launch: n back-to-back launches between one
    pair of CUDA events on the launching stream (the host enqueues faster
    than the kernels run, so launch latency is hidden)."""
    import torch
    for _ in range(warm):
        fn()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(n):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / n  # ms


def bench_pt(steps: int, warmup: int):
    """64^3 x 32 replicas, beta in [0.450, 0.458], 1 + 3 passes, exchange and
    lattice sums every sweep, three ways: every replica batched into each
    half-sweep kernel (CUDA graph), the persistent launches (one per part
    of a sweep, chained, graph-captured), and the plain per-replica launch loop
    (one context per replica, kernels issued replica by replica)."""
    import torch
    from paper_1211_0780_b300 import xy
    L, R, sweeps = 64, 32, 10
    betas = np.linspace(0.450, 0.458, R)
    upd = sweeps * 4 * R * L ** 3
    st = torch.cuda.current_stream()
    out = {"workload": "64^3 x 32 replicas, beta=linspace(0.450,0.458,32), 1+3 passes, exchange+measure every sweep",
           "unit": UNIT}
    for mode, name in ((xy.EXEC_GRAPH, "batched_graph"), (xy.EXEC_PERSISTENT, "batched_persistent")):
        s = xy.Simulation(L, R, betas, SEED, series_capacity=sweeps * (steps + warmup + 4))
        s.set_exec(mode)
        tile = s.autotune(1, 3)[0]
        step = lambda: s.sweep(1, 3, sweeps, measure_every=1, pt_swap_every=1)
        for _ in range(warmup):
            step()
        s.read_series()
        ms = time_kernel(step, st, steps, warm=0)
        s.read_series()
        out[name] = upd / (ms * 1e6)
        out[name + "_tile"] = list(tile)
    reps = [xy.Simulation(L, 1, [b], SEED + i) for i, b in enumerate(betas)]
    for r in reps:
        r.set_tile(0, *out["batched_graph_tile"])

    def one_step():
        for _ in range(sweeps):
            for r in reps:
                r.sweep(1, 3, 1)

    for _ in range(warmup):
        one_step()
    ms_l = time_kernel(one_step, st, max(1, steps // 2), warm=0)
    out["plain_per_replica_loop"] = upd / (ms_l * 1e6)
    return out


RAGGED_L = (16, 24, 32, 48, 64, 96, 128)


def bench_ragged(steps: int, warmup: int):
    """L in {16, 24, 32, 48, 64, 96, 128} x 16 replicas each (beta in
    [0.452, 0.456]), 1 Metropolis + 3 over-relaxation passes, exchange every
    sweep and lattice sums every 10 sweeps, all lattices in the persistent
    launches and, with per-lattice tiles, as a CUDA graph (436 MB
    of (cos, sin) state: HBM-resident).  Also the bandwidth the better
    figure implies against the measured HBM peak, on the metric's 12 B per
    update and on the bytes the chosen tiles move (12 per update on angle
    storage, 24 on vectors)."""
    import torch
    from paper_1211_0780_b300 import xy
    R, sweeps = 16, 10
    betas = np.concatenate([np.linspace(0.452, 0.456, R) for _ in RAGGED_L])
    upd = sweeps * 4 * R * sum(L ** 3 for L in RAGGED_L)
    st = torch.cuda.current_stream()
    s = xy.Simulation(list(RAGGED_L), [R] * len(RAGGED_L), betas, SEED,
                      series_capacity=(steps + warmup + 2) * sweeps)
    s.set_exec(xy.EXEC_PERSISTENT)
    tiles = s.autotune(1, 3)
    out = {"workload": "L in {16,24,32,48,64,96,128} x 16 replicas, 1+3 passes, exchange every sweep, "
                       "sums every 10 sweeps", "unit": UNIT, "tiles": [list(t) for t in tiles]}
    for mode, name in ((xy.EXEC_PERSISTENT, "persistent"), (xy.EXEC_GRAPH, "graph")):
        try:
            s.set_exec(mode)
            if mode == xy.EXEC_GRAPH:  # per-lattice tiles of its own (any kind, per-launch limits)
                out["graph_tiles"] = [list(t) for t in s.autotune(1, 3)]
            for _ in range(warmup):
                s.sweep(1, 3, sweeps, measure_every=10, pt_swap_every=1)
            s.read_series()
            ms = time_kernel(lambda: s.sweep(1, 3, sweeps, measure_every=10, pt_swap_every=1), st, steps, warm=0)
            s.read_series()
            out[name] = upd / (ms * 1e6)
        except Exception as exc:
            out[name] = {"error": repr(exc)}
    hbm, src = measured_peaks()
    figures = {k: out[k] for k in ("persistent", "graph") if isinstance(out.get(k), float)}
    if figures:
        name = max(figures, key=figures.get)
        best = figures[name]
        # bytes each update moves with the chosen tiles: 12 on angle storage
        # (tile kind 4: an angle read and written, the other colour's angle
        # read), 24 on (cos, sin) vectors; averaged over the batch's updates
        kinds = [t[2] for t in (out["graph_tiles"] if name == "graph" else out["tiles"])]
        w = np.array([L ** 3 for L in RAGGED_L], dtype=np.float64)
        moved = float(np.sum(w * np.array([12.0 if k == 4 else 24.0 for k in kinds])) / np.sum(w))
        out["roofline"] = {"bound": "hbm", "unit": "GB/s", "peak": hbm, "peak_source": f"MEASURED_PEAKS.json ({src})",
                           "achieved_12B": best * BYTES_PER_UPDATE, "frac_12B": best * BYTES_PER_UPDATE / hbm,
                           "bytes_moved_per_update": moved,
                           "achieved_moved": best * moved, "frac_moved": best * moved / hbm,
                           "note": f"the {name} figure (the better of the two); the bytes moved per update are "
                                   "12 on angle storage and 24 on the (cos, sin) layout, weighted by each "
                                   "lattice's share of the updates (the 128^3 half-sweeps read exactly their "
                                   "bytes from DRAM: profiles/overrelax_L128x16_direct4x8_dram.md, "
                                   "profiles/angle_L128x16_ncu.md; the angle-storage kernels of L = 96 and 128 "
                                   "take two thirds of the kernel time: "
                                   "profiles/ragged_L16-128x16_launch_list.md)"}
    return out


def bench_reweight(reps: int):
    """Forward + backward reweighting of T = 10^6 samples to K = 4096 beta'
    in [0.4530, 0.4555], one synthetic series per L in {32, 64, 128, 160}."""
    import torch
    from paper_1211_0780_b300 import xy
    from paper_1211_0780_b300.inputs import synthetic_series
    T, K = 10 ** 6, 4096
    st = torch.cuda.current_stream()
    bp = torch.linspace(0.4530, 0.4555, K, dtype=torch.float64, device="cuda")
    total_ms, per_L = 0.0, {}
    for L in (32, 64, 128, 160):
        s = synthetic_series(L, T, 100 + L)
        tens = dict(zip(("E", "m2", "m4", "c", "s2"), xy._series_tensors(s)))
        scratch = torch.empty(xy.lib().xy_reweight_scratch_bytes(T, K), dtype=torch.uint8, device="cuda")
        gU = torch.ones(K, dtype=torch.float64, device="cuda")

        def one():
            f = xy.reweight_forward(tens, 0.4542, bp, L, scratch=scratch)
            xy.reweight_backward(bp, L, f, gU, gU)

        ms = time_kernel(one, st, reps, warm=1)
        per_L[str(L)] = ms
        total_ms += ms
    pairs = 4 * K * T
    # 12 FP64 instructions per (beta', sample) pair: the weight step and the
    # 11 accumulations (1 add + 10 fused multiply-adds by w; the products of
    # e with the observables are formed once per sample and block)
    fp64_ops = 12.0 * pairs
    return {"workload": "4 series (L=32,64,128,160) x T=1e6 samples x K=4096 beta', forward+backward, FP64",
            "pairs_per_ns": pairs / (total_ms * 1e6), "ms_total": total_ms, "ms_per_L": per_L,
            "fp64_instr_per_s": fp64_ops / (total_ms * 1e-3)}


def bench_fss(reps: int):
    """Finite-size-scaling pass: per-bin reweighting sums of 4 synthetic
    series (L = 32, 64, 128, 160; T = 10^6 in 200 bins of 5000) to K = 4096
    beta' in [0.4530, 0.4555], 200 bootstrap resamples of the bins, the
    resampled U_L and rho_s L curves with derivatives, and the crossings of
    consecutive sizes (both observables) with 1/nu from the slopes."""
    import time
    import torch
    from paper_1211_0780_b300 import fss, xy
    from paper_1211_0780_b300.inputs import synthetic_series
    T, K, n_bins, B = 10 ** 6, 4096, 200, 200
    st = torch.cuda.current_stream()
    bp = torch.linspace(0.4530, 0.4555, K, dtype=torch.float64, device="cuda")
    series = {}
    for L in (32, 64, 128, 160):
        s = synthetic_series(L, T, 100 + L)
        series[L] = dict(zip(("E", "m2", "m4", "c", "s2"), xy._series_tensors(s)))
    counts = fss.bootstrap_counts(n_bins, B, seed=12)
    scratch = torch.empty(xy.lib().xy_reweight_bins_scratch_bytes(T, K, n_bins), dtype=torch.uint8, device="cuda")
    stage = {"bin_sums": 0.0, "resample": 0.0, "curves": 0.0, "crossings": 0.0}
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    out = None
    for rep in range(reps + 1):
        ev[0].record(st)
        bins = {L: fss.bin_sums(series[L], 0.4542, bp, n_bins, scratch)[0] for L in series}
        ev[1].record(st)
        sums = {L: fss.resample(bins[L], counts) for L in series}
        ev[2].record(st)
        cur = {L: fss.curves(sums[L], bp, L) for L in series}
        ev[3].record(st)
        Ls = sorted(series)
        out = {f"{a}-{b}-{w}": fss.crossings(bp, a, cur[a], b, cur[b], w)
               for a, b in zip(Ls[:-1], Ls[1:]) for w in ("U", "rhoL")}
        ev[4].record(st)
        torch.cuda.synchronize()
        if rep == 0:
            continue  # warm-up
        for i, key in enumerate(stage):
            stage[key] += ev[i].elapsed_time(ev[i + 1]) / reps
    total = sum(stage.values())
    crossed = {k: int(torch.isfinite(v[:, 0]).sum()) for k, v in out.items()}
    pairs = 4 * K * T
    return {"workload": "4 series (L=32,64,128,160) x T=1e6 in 200 bins x K=4096 beta', 200 bootstrap resamples, "
                        "U_L and rho_s L crossings of consecutive sizes",
            "ms_total": total, "ms_per_stage": stage, "pairs_per_ns": pairs / (stage["bin_sums"] * 1e6),
            "resamples_crossed": crossed}


def bench_ladder():
    """Adaptive ladder: 32^3 x 16 replicas on a linear ladder over
    [0.440, 0.475] (across beta_c), three rounds of 1000 sweeps (1 + 3
    passes, exchange every sweep) each followed by the equal-acceptance
    update; reports the acceptance rates of the first and last ladders and
    the time per round."""
    import time
    import torch
    from paper_1211_0780_b300 import ladder, xy
    L, R = 32, 16
    b0 = np.linspace(0.440, 0.475, R)
    sim = xy.Simulation(L, R, b0, SEED)
    sim.set_exec(xy.EXEC_GRAPH)
    sim.sweep(1, 3, 200, pt_swap_every=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = ladder.adapt(sim, 0, n_iter=3, sweeps=1000, n_metropolis=1, n_overrelax=3, damping=0.7)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    first, last = hist[0][1], hist[-1][1]
    return {"workload": "32^3 x 16 replicas, linear ladder on [0.440, 0.475], 3 rounds x 1000 sweeps (1+3 passes)",
            "ms_per_round": dt * 1e3 / 4, "acceptance_first": [round(float(v), 4) for v in first],
            "acceptance_last": [round(float(v), 4) for v in last],
            "spread_first": float(np.ptp(first)), "spread_last": float(np.ptp(last)),
            "ladder_last": [round(float(v), 5) for v in hist[-1][0]]}


def bench_multihist():
    """Multi-histogram reweighting of a real ladder: 32^3 x 32 replicas on
    beta = linspace(0.440, 0.468, 32), 3000 measured sweeps (1 + 3 passes,
    exchange every sweep) -> 96,000 pooled records; the free energies solved
    to 1e-10 and averages at K = 4096 beta' in [0.440, 0.468]."""
    import time
    import torch
    from paper_1211_0780_b300 import multihist as mh, xy
    L, R, sweeps, K = 32, 32, 3000, 4096
    betas = np.linspace(0.440, 0.468, R)
    sim = xy.Simulation(L, R, betas, SEED, series_capacity=sweeps)
    sim.set_exec(xy.EXEC_GRAPH)
    sim.sweep(1, 3, 500, pt_swap_every=1)
    sim.read_series()
    sim.sweep(1, 3, sweeps, measure_every=1, pt_swap_every=1)
    parts, b = mh.series_from_records(sim.read_series(), L, R)
    pooled, counts = mh.pool(parts)
    pooled = dict(zip(("E", "m2", "m4", "c", "s2"), xy._series_tensors(pooled)))  # resident on the device
    T = int(counts.sum())
    scratch = torch.empty(xy.lib().xy_multihist_scratch_bytes(T, R, K), dtype=torch.uint8, device="cuda")
    mh.solve(pooled, b, counts, tol=1e-6, scratch=scratch)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    f, iters = mh.solve(pooled, b, counts, tol=1e-10, scratch=scratch)
    torch.cuda.synchronize()
    t_solve = time.perf_counter() - t0
    bp = np.linspace(0.440, 0.468, K)
    st = torch.cuda.current_stream()
    ms_fwd = time_kernel(lambda: mh.forward(pooled, b, counts, f, bp, L, scratch=scratch), st, 3, warm=1)
    return {"workload": f"32^3 x 32 replicas, beta=linspace(0.440,0.468,32), {T} pooled records, K=4096 beta'",
            "records": T, "iterations": iters, "ms_solve": t_solve * 1e3, "ms_per_iteration": t_solve * 1e3 / iters,
            "ms_forward": ms_fwd, "exp_per_ns_forward": K * T / (ms_fwd * 1e6)}


def measured_units():
    from paper_1211_0780_b300 import xy
    out = {}
    for k in xy.PEAK_KINDS:
        try:
            out[k] = xy.peak_probe(k)
        except Exception as exc:  # report, do not hide
            out[k] = repr(exc)
    return out


def run_gpu(args):
    import torch
    from paper_1211_0780_b300 import xy
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    st = torch.cuda.current_stream()
    sim = xy.Simulation(L_MAIN, 1, [BETA_MAIN], SEED + rank, series_capacity=args.steps + args.warmup + 4)
    if args.tile:
        parts = [int(v) for v in args.tile.split(",")]
        sim.set_tile(0, *parts)
        tile = sim.get_tile(0)
    else:
        tile = sim.autotune(NM_MAIN, NOR_MAIN)[0]
    sim.set_exec(xy.EXEC_GRAPH)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def step():
        sim.sweep(NM_MAIN, NOR_MAIN, SWEEPS_PER_STEP, measure_every=SWEEPS_PER_STEP)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    sim.read_series()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    clocks = ClockSampler(dev)
    clocks.start()
    if clocks.source and clocks.source.startswith("nvidia-smi"):
        time.sleep(0.3)  # let nvidia-smi start sampling
    for a, b in evs:
        flush.zero_()
        a.record(st)
        step()
        b.record(st)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    ms_local = sum(step_ms)
    ms_total = allreduce_max(ms_local, world)
    recs = sim.read_series()
    assert len(recs) == args.steps and np.all(np.isfinite(recs["E"]))
    value = world * args.steps * UPDATES_PER_STEP / (ms_total * 1e6)
    launches_per_step = SWEEPS_PER_STEP * (NM_MAIN + NOR_MAIN) * 2 + 2  # half-sweeps + finish + advance

    # Four more runs of the same K steps (same flush, same events), after the
    # timed region: the median of the five runs, as context beside `value`.
    runs = [value]
    for _ in range(4):
        ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        barrier(world)
        torch.cuda.synchronize()
        for a, b in ev2:
            flush.zero_()
            a.record(st)
            step()
            b.record(st)
        torch.cuda.synchronize()
        barrier(world)
        ms_r = allreduce_max(sum(a.elapsed_time(b) for a, b in ev2), world)
        runs.append(world * args.steps * UPDATES_PER_STEP / (ms_r * 1e6))
        assert len(sim.read_series()) == args.steps  # one record per step, drained per run

    # --- per-kernel durations (CUDA events on the launching stream) ----------
    # Graph-captured runs of one pass type, each one CUDA graph (the library
    # captures up to 16 sweeps per graph): 16 sweeps of 0 + 5 passes = 160
    # over-relaxation half-sweeps, 16 sweeps of 1 + 0 = 32 Metropolis ones
    # (plus one counter-advance kernel each), replayed back to back.  Average
    # per half-sweep, including the kernel-to-kernel gaps of the graph.
    ms_or = time_kernel(lambda: sim.sweep(0, 5, 16), st, 5) / 160
    ms_met = time_kernel(lambda: sim.sweep(1, 0, 16), st, 20) / 32
    half = L_MAIN ** 3 // 2
    hbm, src = measured_peaks()
    ach = BYTES_PER_UPDATE * half / (ms_or * 1e-3) / 1e9
    # DRAM bytes per launch from the committed ncu capture of this tile's
    # over-relaxation kernel (valid only for the tile that capture used)
    traffic, traffic_note, l2_bytes = None, "no ncu capture for this tile", None
    kind_names = {0: "march", 1: "block", 2: "stream", 3: "direct"}
    tile_name = f"{kind_names.get(tile[2], tile[2])}{tile[0]}x{tile[1]}"
    prof = os.path.join(ROOT, "profiles", f"overrelax_L160_{tile_name}_traffic.txt")
    if os.path.exists(prof):
        kv = {}
        with open(prof) as f:
            for line in f:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("tile") == ",".join(str(v) for v in tile):
            traffic = int(kv["dram_bytes_per_launch"])
            l2_bytes = int(kv["l2_read_bytes_per_launch"]) if "l2_read_bytes_per_launch" in kv else None
            traffic_note = (f"cold-cache ncu capture (profiles/overrelax_L160_{tile_name}_traffic.txt, "
                            f"profiles/overrelax_L160_{tile_name}_ncu.md): the whole "
                            "(cos, sin) state read once, 8 B per site against the 4 B per site of the "
                            "12 B/update angle figure")
    roofline = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "traffic": traffic, "traffic_note": traffic_note,
                "kernel": ("k_half_direct" if tile[2] == 3 else "k_half") + "<over-relaxation>, 160^3 half-sweep, "
                          f"{tile_name} tile",
                "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({src})",
                "note": ("12 B/update algorithmic; lattice state (cos, sin) is L2-resident (32.8 MB < 126 MB); "
                         "duration = CUDA-event average over 5 back-to-back replays of a graph of 160 "
                         "chained over-relaxation half-sweeps (+1 counter kernel)")}
    # the same 12 B/update basis over the Metropolis half-sweep and over the
    # whole timed step (every kernel of the 10 sweeps, the fused sums and the
    # finishing step, and the gaps between them)
    ach_met = BYTES_PER_UPDATE * half / (ms_met * 1e-3) / 1e9
    ach_step = BYTES_PER_UPDATE * UPDATES_PER_STEP / (ms_total / args.steps * 1e-3) / 1e9
    roofline["metropolis"] = {"achieved": ach_met, "frac": ach_met / hbm, "unit": "GB/s",
                              "kernel": "Metropolis half-sweep, same tile and timing as above"}
    roofline["step"] = {"achieved": ach_step, "frac": ach_step / hbm, "unit": "GB/s",
                        "note": "12 B x updates per step / ms_per_step: the whole 1 + 5 step"}
    kernels = {"overrelax_half_ms": ms_or, "metropolis_half_ms": ms_met,
               "overrelax_updates_per_ns": half / (ms_or * 1e6), "metropolis_updates_per_ns": half / (ms_met * 1e6)}

    # --- end to end through the C-ABI with host buffers --------------------
    # Each step uploads its input state as FP32 angles (4 B per site, the
    # method's own representation; converted to (cos, sin) on the device),
    # sweeps, and reads the step's measurement record back.  Serial: one
    # simulation, upload -> sweeps -> read.  Pipelined (the reported value):
    # two simulations of the same lattice on two streams take the steps in
    # turn, so the upload of step k+1 (copy engine) overlaps the sweeps of
    # step k (SMs); an event keeps the sweeps of consecutive steps from
    # overlapping one another, so the figure gains only the hidden copies.
    # The first step's upload has no sweeps to hide behind (the pipeline's
    # fill): twice the device-timed step count spreads it as a long job would.
    e2e_steps = max(8, 2 * args.steps)
    n_ang = sim.n_packed_angles()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    sims = []
    for i, s_ in enumerate(streams):
        e = xy.Simulation(L_MAIN, 1, [BETA_MAIN], SEED + rank + 7 * (i + 1), series_capacity=e2e_steps + 8,
                          stream=s_)
        e.set_tile(0, *tile)
        e.set_exec(xy.EXEC_GRAPH)
        sims.append(e)
    # page-locked host buffers from the library (xy_host_alloc)
    pinned = [xy.pinned_empty(n_ang), xy.pinned_empty(n_ang)]
    sim.get_packed_angles(pinned[0])
    pinned[1][:] = pinned[0]
    for e, hb in zip(sims, pinned):  # warm-up: graphs captured, series drained
        e.set_packed_angles(hb)
        e.sweep(NM_MAIN, NOR_MAIN, SWEEPS_PER_STEP, measure_every=SWEEPS_PER_STEP)
        e.read_series()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        sims[0].set_packed_angles(pinned[0])  # H2D of the step's input state (pinned)
        sims[0].sweep(NM_MAIN, NOR_MAIN, SWEEPS_PER_STEP, measure_every=SWEEPS_PER_STEP)
        r = sims[0].read_series()             # D2H of the step's measurement (synchronises)
    t_serial = time.perf_counter() - t0
    done = [torch.cuda.Event(), torch.cuda.Event()]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        i = k % 2
        sims[i].set_packed_angles(pinned[i])  # waits for this stream's copy only
        if k > 0:
            streams[i].wait_event(done[1 - i])
        sims[i].sweep(NM_MAIN, NOR_MAIN, SWEEPS_PER_STEP, measure_every=SWEEPS_PER_STEP)
        done[i].record(streams[i])
        if k > 0:
            r = sims[1 - i].read_series()     # previous step's record (synchronises its stream)
            assert len(r) == 1
    r = sims[(e2e_steps - 1) % 2].read_series()
    t_e2e = time.perf_counter() - t0
    assert len(r) == 1 and np.all(np.isfinite(r["E"]))
    # the upload alone (copy + on-device conversion), CUDA events on its stream
    ua, ub = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ua.record(streams[0])
    for _ in range(5):
        sims[0].set_packed_angles(pinned[0])
    ub.record(streams[0])
    ub.synchronize()
    ms_up = ua.elapsed_time(ub) / 5
    e2e = {"value": world * e2e_steps * UPDATES_PER_STEP / (t_e2e * 1e9), "unit": UNIT,
           "h2d_bytes_per_step": int(n_ang * 4), "d2h_bytes_per_step": int(r.nbytes),
           "input": "FP32 angles of the 160^3 lattice, packed order, page-locked host memory (xy_host_alloc)",
           "pipelined": "two simulations on two streams take alternate steps; step k+1's upload overlaps "
                        "step k's sweeps, the sweeps of consecutive steps never overlap",
           "steps": e2e_steps,
           "serial_value": world * e2e_steps * UPDATES_PER_STEP / (t_serial * 1e9),
           "upload_ms": ms_up, "upload_gbs": n_ang * 4 / (ms_up * 1e6), "sweeps_ms": ms_total / args.steps,
           "bound": "host-to-device link (the upload is longer than the sweeps)" if ms_up > ms_total / args.steps
                    else "sweeps (the upload is hidden behind them)"}
    torch.cuda.synchronize()
    del sims

    extras = {}
    if not args.no_extras and rank == 0:
        for key, fn in (("batched_pt", lambda: bench_pt(max(3, args.steps // 2), 2)),
                        ("ragged", lambda: bench_ragged(max(3, args.steps // 4), 2)),
                        ("reweight", lambda: bench_reweight(3)),
                        ("fss", lambda: bench_fss(3)),
                        ("ladder", bench_ladder),
                        ("multihist", bench_multihist),
                        ("units", measured_units)):
            try:
                extras[key] = fn()
            except Exception as exc:  # report, do not hide
                extras[key] = {"error": repr(exc)}
        if isinstance(extras.get("reweight"), dict) and isinstance(extras.get("units"), dict):
            peak = extras["units"].get("fp64_fma")
            if isinstance(peak, float):
                extras["reweight"]["roofline"] = {
                    "bound": "alu", "unit": "FP64 instr/s", "achieved": extras["reweight"]["fp64_instr_per_s"],
                    "peak": peak, "frac": extras["reweight"]["fp64_instr_per_s"] / peak,
                    "peak_source": "xy_peak_probe FP64 FMA (measured here)"}
    # context for the L2-resident state: the kernel's L2 -> L1 read bytes (ncu,
    # warm) over its duration, against the measured L2 read bandwidth
    l2_peak = extras.get("units", {}).get("l2_read_bytes") if isinstance(extras.get("units"), dict) else None
    if l2_bytes and isinstance(l2_peak, float):
        l2_ach = l2_bytes / (ms_or * 1e-3) / 1e9
        roofline["l2"] = {"achieved": l2_ach, "peak": l2_peak / 1e9, "unit": "GB/s", "frac": l2_ach * 1e9 / l2_peak,
                          "source": "L2->L1 read bytes per launch from a warm ncu capture; peak: xy_peak_probe "
                                    "L2 read (measured here)"}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        v, n, done = oracle_rate(args.cpu_seconds)
        v1, _, done1 = oracle_rate(min(4.0, args.cpu_seconds), threads=1, sweeps=1)
        cpu = {"value": v, "unit": UNIT, "cores": n, "kind": "oracle",
               "sample": f"{done // SWEEPS_PER_STEP} steps ({done} sweeps of 1+5 passes, lattice sums every "
                         f"{SWEEPS_PER_STEP}) of the 160^3 lattice, FP64, OpenMP over sites",
               "cpu_model": cpu_model(),
               "single_thread": {"value": v1, "unit": UNIT,
                                 "sample": f"{done1} unmeasured sweep{'s' if done1 > 1 else ''} on one thread"}}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_total / args.steps,
            "step_ms": {"median": statistics.median(step_ms), "min": min(step_ms), "max": max(step_ms),
                        "note": "this rank's per-step CUDA-event times"},
            "runs": {"values": runs, "median": statistics.median(runs),
                     "note": "value is the first run; four more runs of the same K steps follow it"},
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(world),
            "tile": list(tile), "exec": "cuda graph of half-sweep kernels",
            "roofline": roofline, "kernels": kernels, "cpu_baseline": cpu, "clocks": clk, "e2e": e2e,
            "gpu_launches": args.steps * launches_per_step,
        }
        line.update(extras)
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--tile", default="", help="ty,tz[,kind] of the 160^3 tile (skips the autotuner)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
