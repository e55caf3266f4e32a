"""A small, fixed launch sequence of one half-sweep kernel, for profilers.

python -m paper_1211_0780_b300.profile_case --L 160 --ty 8 --tz 2 --kind 1 --mode or --launches 5

Creates one lattice (seeded hot start), runs a few warm-up sweeps, then
issues `--launches` half-sweeps of the chosen kernel (or = over-relaxation,
met = Metropolis, meas = measurement-only; sweep = 1 + 5 sweeps; pt = sweeps of
1 + 3 passes with sums and an exchange, the ladder spaced on [0.450, 0.458];
ragged = sweeps of 1 + 3 passes with an exchange, sums every 10 sweeps, on the
lattices L = 16, 24, 32, 48, 64, 96, 128 x 16 replicas each, ladders on
[0.452, 0.456], with the fixed tiles of RAGGED_TILES)
and synchronises (--exec picks plain launches, the CUDA graph or the persistent launches
for the sweep and pt modes); reweight =
`--launches` forward reweightings of one synthetic series of `--T` samples to
`--K` couplings.  No autotuning,
so the launch list is short and deterministic.
"""

import argparse

import numpy as np

# ragged mode: (L, (ty, tz, kind) for the CUDA graph, (ty, tz, kind) for the
# persistent launches, which take one kind for every lattice) -- tiles the
# autotuner picked for these lattices on B300
RAGGED_TILES = ((16, (16, 4, 1), (16, 2, 4)), (24, (8, 8, 1), (12, 2, 4)), (32, (16, 2, 3), (16, 2, 4)),
                (48, (24, 4, 3), (8, 8, 4)), (64, (16, 8, 3), (8, 8, 4)), (96, (8, 8, 4), (4, 32, 4)),
                (128, (8, 16, 4), (4, 32, 4)))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, default=160)
    ap.add_argument("--R", type=int, default=1)
    ap.add_argument("--ty", type=int, default=0)
    ap.add_argument("--tz", type=int, default=0)
    ap.add_argument("--kind", type=int, default=1,
                    help="0 = march, 1 = block, 2 = stream, 3 = direct, 4 = angle storage")
    ap.add_argument("--mode", default="or", choices=["or", "met", "meas", "sweep", "pt", "ragged", "reweight"])
    ap.add_argument("--T", type=int, default=200000, help="samples of the reweight mode's series")
    ap.add_argument("--K", type=int, default=4096, help="couplings of the reweight mode")
    ap.add_argument("--launches", type=int, default=5)
    ap.add_argument("--warm-sweeps", type=int, default=2)
    ap.add_argument("--exec", type=int, default=0,
                    help="execution mode of the sweep and pt modes: 0 plain launches, 1 CUDA graph, 2 persistent")
    args = ap.parse_args()
    import torch
    from paper_1211_0780_b300 import xy
    if args.mode == "reweight":
        # forward reweighting of one synthetic series (L sets its scale)
        from paper_1211_0780_b300.inputs import synthetic_series
        s = synthetic_series(args.L, args.T, 100 + args.L)
        tens = dict(zip(("E", "m2", "m4", "c", "s2"), xy._series_tensors(s)))
        bp = torch.linspace(0.4530, 0.4555, args.K, dtype=torch.float64, device="cuda")
        for _ in range(args.launches):
            xy.reweight_forward(tens, 0.4542, bp, args.L)
        torch.cuda.synchronize()
        print("reweight done")
        return
    if args.mode == "ragged":
        R = 16
        Ls = [t[0] for t in RAGGED_TILES]
        sim = xy.Simulation(Ls, [R] * len(Ls), np.concatenate([np.linspace(0.452, 0.456, R) for _ in Ls]),
                            0x5EED2012, series_capacity=args.warm_sweeps + args.launches + 2)
        for i, t in enumerate(RAGGED_TILES):
            sim.set_tile(i, *(t[2] if args.exec == 2 else t[1]))
        sim.sweep(1, 1, args.warm_sweeps)
        sim.set_exec(args.exec)
        for _ in range(args.launches):
            sim.sweep(1, 3, 1, measure_every=10, pt_swap_every=1)
        torch.cuda.synchronize()
        print("ragged done")
        return
    betas = (np.linspace(0.450, 0.458, args.R) if args.mode == "pt" else np.linspace(0.4542, 0.4560, args.R)) \
        if args.R > 1 else [0.4542]
    sim = xy.Simulation(args.L, args.R, betas, 0x5EED2012)
    if args.ty and args.tz:
        sim.set_tile(0, args.ty, args.tz, args.kind)
    sim.sweep(1, 1, args.warm_sweeps)
    sim.set_exec(args.exec)
    for i in range(args.launches):
        if args.mode == "or":
            sim.overrelax_half(i & 1)
        elif args.mode == "met":
            sim.metropolis_half(i & 1, 1000 + i)
        elif args.mode == "meas":
            sim.measure()
        elif args.mode == "pt":
            # one sweep of 1 + 3 passes with the sums and an exchange (the PT workload)
            sim.sweep(1, 3, 1, measure_every=1, pt_swap_every=1)
        else:
            sim.sweep(1, 5, 1)
    torch.cuda.synchronize()
    print("tile", sim.get_tile(0), "done")


if __name__ == "__main__":
    main()
