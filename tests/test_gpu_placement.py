"""Blocks of one continuous-scale domain placed on several ranks, on the GPU through the
C-ABI: a step run phase by phase (lbm_step_phase) is bit for bit lbm_step; ranks that each
compute only their own blocks and exchange the node boxes of the plan (lbm_pack_box /
lbm_unpack_box) reproduce the undivided domain bit for bit on every owned block, held by
one process or by two processes exchanging through torch.distributed; the library's
mapping boxes are the ones the oracle-based plan test uses."""
import os
import socket

import numpy as np
import pytest
import torch

import synth
from paper_1807_02284_gb300 import sharding
from tests.helpers import f32

pytestmark = pytest.mark.gpu


def _scene():
    return synth.multiscale(scale=0.25, nu=2e-3, flow_amp=0.06)


def _domain(sc, stream=None):
    from paper_1807_02284_gb300 import lbm
    b0 = sc.blocks[0]
    dom = lbm.Domain(b0.dims, sc.nu, periodic=sc.periodic, adaptive=sc.adaptive,
                     c_src=sc.c_src, stream=stream)
    for b in sc.blocks[1:]:
        dom.add_scale_block(b.origin, b.h, b.dims)
    for i, b in enumerate(sc.blocks):
        dom.set_flags(b.flags, block=i)
        dom.init_macro(f32(b.u0), rho=f32(b.rho0), c=f32(b.c0), block=i)
    return dom


def _state(dom, b):
    from paper_1807_02284_gb300 import lbm
    return [dom.read_field(fld, lbm.LBM_F32, b) for fld in
            (lbm.LBM_FIELD_F, lbm.LBM_FIELD_U, lbm.LBM_FIELD_SCALAR)]


def _undivided(steps):
    dom = _domain(_scene())
    for _ in range(steps):
        dom.step(1)
    out = [_state(dom, b) for b in range(3)]
    dom.close()
    return out


def test_phased_step_equals_lbm_step(lib):
    from paper_1807_02284_gb300 import lbm
    want = _undivided(3)
    dom = _domain(_scene())
    one = sharding.PlacedDomain(dom, [0, 0, 0], 0)
    sharding.step_placed_local([one], 3)
    for b in range(3):
        for x, y in zip(_state(dom, b), want[b]):
            assert np.array_equal(x, y), b
    assert dom.info(0).steps == 3
    dom.close()


@pytest.mark.parametrize("owner", [[0, 1, 1], [0, 0, 1], [1, 0, 2]])
def test_placed_blocks_reproduce_lbm_step(lib, owner):
    steps = 3
    want = _undivided(steps)
    stream = torch.cuda.Stream()
    ranks = [sharding.PlacedDomain(_domain(_scene(), stream), owner, r)
             for r in range(max(owner) + 1)]
    sharding.step_placed_local(ranks, steps)
    for r in ranks:
        r.sync()
        for b, o in enumerate(owner):
            if o == r.rank:
                for x, y in zip(_state(r.dom, b), want[b]):
                    assert np.array_equal(x, y), (owner, r.rank, b)
    for r in ranks:
        r.dom.close()


def test_library_boxes_match_the_plan_geometry(lib):
    from paper_1807_02284_gb300 import lbm
    from tests.placed_oracle import OraclePlacedDomain
    sc = _scene()
    dom = _domain(sc)
    ref = OraclePlacedDomain(sc)
    for b in (1, 2):
        p = dom.info(b).parent
        assert p == ref.info(b).parent
        assert dom.mapping_boxes(b, lbm.LBM_BOX_PRIOR_SOURCE, p) == \
            ref.mapping_boxes(b, lbm.LBM_BOX_PRIOR_SOURCE, p)
        for k in range(3):
            if k != b:
                assert dom.mapping_boxes(b, lbm.LBM_BOX_POST_TARGET, k) == \
                    ref.mapping_boxes(b, lbm.LBM_BOX_POST_TARGET, k), (b, k)
    dom.close()


def test_phase_and_box_argument_checks(lib):
    from paper_1807_02284_gb300 import lbm
    dom = _domain(_scene())
    buf = torch.empty(dom.box_bytes(0, (0, 0, 0), (3, 3, 3)), dtype=torch.uint8, device="cuda")
    with pytest.raises(lbm.LBMError) as ei:               # start level outside a phased step
        dom.pack_box(0, lbm.LBM_LEVEL_START, (0, 0, 0), (3, 3, 3), buf)
    assert ei.value.status == lbm.LBM_ERR_STATE
    assert dom.box_bytes(0, (0, 0, 0), (32, 3, 3)) == 0   # outside the 32^3 block
    with pytest.raises(lbm.LBMError) as ei:
        dom.step_phase(lbm.LBM_PHASE_REFERENCE)           # before BEGIN
    assert ei.value.status == lbm.LBM_ERR_STATE
    dom.step_phase(lbm.LBM_PHASE_BEGIN)
    dom.pack_box(0, lbm.LBM_LEVEL_START, (0, 0, 0), (3, 3, 3), buf)
    with pytest.raises(lbm.LBMError) as ei:
        dom.step_phase(lbm.LBM_PHASE_BLOCK, 1)            # before the reference phase
    assert ei.value.status == lbm.LBM_ERR_STATE
    dom.step_phase(lbm.LBM_PHASE_REFERENCE)
    with pytest.raises(lbm.LBMError) as ei:
        dom.step_phase(lbm.LBM_PHASE_BLOCK, 2)            # out of order
    assert ei.value.status == lbm.LBM_ERR_STATE
    with pytest.raises(lbm.LBMError) as ei:
        dom.step_phase(lbm.LBM_PHASE_BLOCK, 0)            # not a refined block
    assert ei.value.status == lbm.LBM_ERR_INVALID_ARG
    with pytest.raises(lbm.LBMError) as ei:
        dom.step_phase(lbm.LBM_PHASE_END)                 # blocks not done
    assert ei.value.status == lbm.LBM_ERR_STATE
    for b in (1, 2):
        dom.step_phase(lbm.LBM_PHASE_BLOCK, b)
        dom.step_phase(lbm.LBM_PHASE_POST, b)
    dom.step_phase(lbm.LBM_PHASE_END)
    dom.sync()
    dom.close()
    far = synth.random_scene(dims=(12, 12, 12), seed=3, periodic=(False,) * 3)
    fb = synth.far_block(far.blocks[0], 2.0, 4.0)
    d2 = lbm.Domain((12, 12, 12), 0.01)
    d2.add_scale_block(fb.origin, fb.h, fb.dims)
    with pytest.raises(lbm.LBMError) as ei:
        d2.step_phase(lbm.LBM_PHASE_BEGIN)
    assert ei.value.status == lbm.LBM_ERR_UNSUPPORTED
    d2.close()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _gloo_worker(rank, world, port, owner, steps, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r = sharding.PlacedDomain(_domain(_scene()), owner, rank)
        r.step(steps)
        r.sync()
        q.put((rank, {b: _state(r.dom, b) for b, o in enumerate(owner) if o == rank}))
        r.dom.close()
    finally:
        dist.barrier()
        dist.destroy_process_group()


def test_two_process_placement_through_torch_distributed(lib):
    """Two processes on the same GPU, the boxes moving through gloo (staged through host
    memory), so no kernel of one process waits for the other."""
    import torch.multiprocessing as mp
    owner, steps = [0, 1, 1], 3
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gloo_worker, args=(r, 2, port, owner, steps, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    want = _undivided(steps)
    for rank, blocks in res.items():
        for b, fields in blocks.items():
            for x, y in zip(fields, want[b]):
                assert np.array_equal(x, y), (rank, b)
