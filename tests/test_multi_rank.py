"""Multi-rank logic on CPU (gloo, world size 2).

The path shards only as independent replicas (weak scaling): every rank hulls
its own set, and bench.py reduces the timed region with a max over ranks. The
shard identity below is what a real shard-and-merge of one set would rely on:
the hood of a union is the hood of the union of the shards' hoods.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
import oracle
from paper_1203_5004_gb300 import inputs


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n, ret):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # max over ranks of a per-rank time (bench.py's timing reduction)
        mine = 1.5 + rank
        got_max = bench.max_over_ranks(mine, dist, "cpu")
        # weak scaling: every rank has its own seed and set
        seed = bench.rank_seed(7, rank)
        # shard identity: ranks hull contiguous shards of one set
        full = inputs.uniform(n, 123)
        lo, hi = rank * n // world, (rank + 1) * n // world
        h = oracle.upper_hull(full.kx[lo:hi], full.ky[lo:hi]) + lo
        parts = [None] * world
        dist.all_gather_object(parts, h.tolist())
        if rank == 0:
            cand = np.array(sum(parts, []), dtype=np.int64)
            sub = oracle.upper_hull(full.kx[cand], full.ky[cand])
            merged = cand[sub].tolist()
            ret.put((got_max, seed, merged, oracle.upper_hull(full.kx, full.ky).tolist()))
        else:
            ret.put((got_max, seed, None, None))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, 20000, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    maxes = sorted(r[0] for r in res)
    assert maxes == [2.5, 2.5]
    seeds = sorted(r[1] for r in res)
    assert seeds == [7, 1007]
    merged = [r for r in res if r[2] is not None][0]
    assert merged[2] == merged[3]


def test_max_over_ranks_without_group():
    assert bench.max_over_ranks(3.25) == 3.25
