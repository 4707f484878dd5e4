"""Blocks of one continuous-scale domain placed on several ranks (no counterpart in the
paper): the exchange plan and the phase order, checked on CPU with the FP64 oracle behind
the placement's domain interface -- ranks that each compute only their own blocks and
exchange the node boxes of the plan reproduce the undivided domain exactly."""
import numpy as np
import pytest
import torch

import synth
from oracle import coupling
from paper_1807_02284_gb300 import lbm, sharding
from tests.placed_oracle import OraclePlacedDomain


def _scene():
    return synth.multiscale(scale=0.25, nu=2e-3, flow_amp=0.06)


def _ranks(owner):
    world = max(owner) + 1
    return [sharding.PlacedDomain(OraclePlacedDomain(_scene()), owner, r) for r in range(world)]


def _assert_owned_equal(ranks, ref, exact=True):
    for r in ranks:
        for b, o in enumerate(r.owner):
            if o != r.rank:
                continue
            a, e = r.dom.ms.blocks[b].state, ref.blocks[b].state
            for x, y in ((a.f, e.f), (a.u, e.u), (a.c, e.c)):
                if exact:
                    assert torch.equal(x, y), (r.rank, b)
                else:
                    assert float((x - y).abs().max()) < 1e-13, (r.rank, b)


def test_phased_step_is_the_oracle_step():
    ref = coupling.MultiScale.build(_scene())
    one = _ranks([0, 0, 0])
    for _ in range(2):
        ref.step()
        sharding.step_placed_local(one, 1)
    assert one[0].moves == []
    _assert_owned_equal(one, ref)


def test_block_placement_plan():
    """Moves of the 3-block scene with s0 alone and s1, s2 together: s1's source boxes of
    both levels (6 faces each) come from rank 0; s1's post-mapping box of s0 goes back; s2
    needs nothing from outside its rank."""
    d = OraclePlacedDomain(_scene())
    r = sharding.PlacedDomain(d, [0, 1, 1], 1)
    stages = {}
    for m in r.moves:
        stages.setdefault(m.stage, []).append(m)
    assert set(stages) == {("prior", 1), ("post", 1), ("post", 2)}
    assert len(stages[("prior", 1)]) == 12
    assert {m.level for m in stages[("prior", 1)]} == {lbm.LBM_LEVEL_START, lbm.LBM_LEVEL_CURRENT}
    assert all((m.src, m.dst, m.block) == (0, 1, 0) for m in stages[("prior", 1)])
    assert [(m.src, m.dst, m.block) for m in stages[("post", 1)]] == [(1, 0, 0)]
    assert [(m.src, m.dst, m.block) for m in stages[("post", 2)]] == [(1, 0, 0)]
    assert sharding.place_blocks([4, 2, 3], 2) == [0, 1, 1]


@pytest.mark.parametrize("owner", [[0, 1, 1], [0, 1, 0], [0, 0, 1], [1, 0, 2]])
def test_placed_blocks_reproduce_the_undivided_domain(owner):
    ref = coupling.MultiScale.build(_scene())
    ranks = _ranks(owner)
    for _ in range(2):
        ref.step()
        sharding.step_placed_local(ranks, 1)
        _assert_owned_equal(ranks, ref)


def test_a_missing_move_breaks_it():
    """Negative control: without the post-mapping boxes sent back, the owner of s0 keeps
    stale values where the finer blocks' interiors should have been mapped in."""
    ref = coupling.MultiScale.build(_scene())
    ranks = _ranks([0, 1, 1])
    for r in ranks:
        r.moves = [m for m in r.moves if m.stage[0] != "post"]
    ref.step()
    sharding.step_placed_local(ranks, 1)
    d = float((ranks[0].dom.ms.blocks[0].state.f - ref.blocks[0].state.f).abs().max())
    assert d > 1e-6


def _gloo_worker(rank, world, port, owner, steps, q):
    import os
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r = sharding.PlacedDomain(OraclePlacedDomain(_scene()), owner, rank)
        r.step(steps)
        out = {b: (r.dom.ms.blocks[b].state.f.numpy(), r.dom.ms.blocks[b].state.c.numpy())
               for b, o in enumerate(owner) if o == rank}
        q.put((rank, out))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("owner", [[0, 1, 1], [1, 0, 1]])
def test_placed_blocks_over_gloo_ranks(owner):
    """Two processes, each computing its blocks and exchanging the boxes through
    torch.distributed (gloo): every owned block equals the undivided oracle's."""
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    steps = 2
    procs = [ctx.Process(target=_gloo_worker, args=(r, 2, port, owner, steps, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=600) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    ref = coupling.MultiScale.build(_scene())
    ref.run(steps)
    for rank, blocks in res.items():
        for b, (f, c) in blocks.items():
            assert owner[b] == rank
            assert np.array_equal(f, ref.blocks[b].state.f.numpy()), (rank, b)
            assert np.array_equal(c, ref.blocks[b].state.c.numpy()), (rank, b)
    assert sorted(b for blocks in res.values() for b in blocks) == [0, 1, 2]
