"""The N>1 host logic of bench.py on CPU with the gloo backend (world size 2):
every rank runs an independent replica, the timed region is bracketed by a
barrier, and the reported time is the maximum over ranks."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    w, r, lr = bench.dist_env()
    assert (w, r, lr) == (world, rank, rank)
    bench.barrier(world)
    t = bench.allreduce_max(10.0 + 5.0 * rank, world)
    seeds = [None] * world
    dist.all_gather_object(seeds, bench.SEED + rank)
    q.put((rank, t, seeds))
    dist.destroy_process_group()


def test_bench_max_over_ranks_and_distinct_replicas():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, seeds in out:
        assert t == 15.0                      # the slower rank's time
        assert len(set(seeds)) == 2           # independent replicas
