"""Multi-process placement of the batched simulations, on CPU with the gloo backend
(world size 2): every simulation runs on exactly one rank, loads are balanced, and the
timing reduction takes the slowest rank and the total work."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import synth
from paper_1807_02284_gb300 import sharding


def test_greedy_placement_is_complete_and_balanced():
    sizes = [s.blocks[0].flags.size for s in synth.batch(64, seed=4)]
    for world in (1, 2, 4, 8):
        shards = sharding.shard_by_cells(sizes, world)
        flat = sorted(i for s in shards for i in s)
        assert flat == list(range(64))
        loads = [sum(sizes[i] for i in s) for s in shards]
        assert max(loads) <= 1.1 * (sum(sizes) / world) + max(sizes) * (world > 8)
    assert sharding.shard_by_cells([5, 3, 3, 1], 2) == [[0, 3], [1, 2]]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sizes = [s.blocks[0].flags.size for s in synth.batch(64, seed=4)]
    mine = sharding.rank_share(sizes, rank, world)
    work = float(sum(sizes[i] for i in mine))
    t_max, w_tot = sharding.reduce_timing(1.0 + rank, work)
    got = [None] * world
    dist.all_gather_object(got, mine)
    q.put((rank, t_max, w_tot, got))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_sharding_and_timing():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sizes = [s.blocks[0].flags.size for s in synth.batch(64, seed=4)]
    for rank, t_max, w_tot, got in res:
        assert t_max == 2.0                       # the slower rank sets the time
        assert w_tot == float(sum(sizes))         # all simulations counted once
        flat = sorted(i for s in got for i in s)
        assert flat == list(range(64))
