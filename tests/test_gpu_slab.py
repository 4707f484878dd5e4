"""A domain cut into slabs along z, with the halo exchange of the plane pack / unpack entry
points before every step, reproduces the undivided domain bit for bit on every owned node:
populations as stored, velocity, scalar and flags.  The cuts cross obstacles (halfway
bounce-back and regularized surfaces), a scalar source and, with open z, the wall faces."""
import os
import socket

import numpy as np
import pytest

import synth
from tests.helpers import f32

pytestmark = pytest.mark.gpu


def _scene(periodic, dims=(20, 18, 21)):
    nz = dims[2]
    sc = synth.random_scene(dims=dims, seed=71, periodic=periodic, nu=0.002,
                            spheres=[(7.0, 8.0, nz / 3, 3.5), (13.0, 10.0, 2 * nz / 3, 3.0)],
                            inflow=(9, 10, 3.0, 0.08))
    b = sc.blocks[0]
    b.flags[nz // 2 - 1:nz // 2 + 1, 3:5, 10:12] |= synth.SCALAR_SRC
    return sc


def _fields(read):
    from paper_1807_02284_gb300 import lbm
    return {k: read(f, d) for k, f, d in (("f", lbm.LBM_FIELD_F, lbm.LBM_F32),
                                          ("u", lbm.LBM_FIELD_U, lbm.LBM_F32),
                                          ("c", lbm.LBM_FIELD_SCALAR, lbm.LBM_F32),
                                          ("flags", lbm.LBM_FIELD_FLAGS, lbm.LBM_U8))}


def _undivided(sc, steps, walls, obstacles, **kw):
    from paper_1807_02284_gb300 import lbm
    b = sc.blocks[0]
    dom = lbm.Domain(b.dims, sc.nu, periodic=sc.periodic, adaptive=sc.adaptive, **kw)
    dom.set_flags(b.flags)
    if walls is not None:
        dom.set_walls(walls, obstacles=obstacles)
    dom.init_macro(f32(b.u0), rho=f32(b.rho0), c=f32(b.c0))
    dom.step(steps)
    nx, ny, nz = b.dims

    def read(field, dt):
        a = dom.read_field(field, dt)
        return a.reshape((a.size // (nx * ny * nz), nz, ny, nx))
    out = _fields(read)
    dom.close()
    return out


def _slab(sc, rank, world, walls, obstacles, **kw):
    from paper_1807_02284_gb300 import sharding
    b = sc.blocks[0]
    s = sharding.SlabDomain(b.dims, sc.nu, rank=rank, world=world, periodic=sc.periodic,
                            adaptive=sc.adaptive, **kw)
    s.set_flags(b.flags)
    if walls is not None:
        s.set_walls(walls, obstacles=obstacles)
    s.init_macro(f32(b.u0), rho=f32(b.rho0), c=f32(b.c0))
    return s


def _owned(s):
    nx, ny, _ = s.dims

    def read(field, dt):
        a = s.dom.read_field(field, dt)
        return s.owned(a.reshape((a.size // (nx * ny * s.plan.local_nz), s.plan.local_nz, ny, nx)))
    return _fields(read)


NEAR_SOLID, OBST_WALL = 16, 64


def _assert_same(parts, want):
    for k, w in want.items():
        got = np.concatenate([p[k] for p in parts], axis=1)
        assert got.shape == w.shape
        if k == "flags":
            # the near-obstacle bit of a regularized surface node is never read (such a node
            # takes no bounce-back) and, next to a cut, may be derived from a halo voxel
            # whose own surface status depends on nodes beyond the slab
            unused = ((w & OBST_WALL) != 0) & ((got & OBST_WALL) != 0)
            keep = np.uint8(0xFF ^ NEAR_SOLID)
            got = np.where(unused, got & keep, got)
            w = np.where(unused, w & keep, w)
        bad = np.argwhere(got != w)
        assert bad.size == 0, (k, bad[:5])


@pytest.mark.parametrize("case", [
    # periodic z: every slab has both halos, the ring wraps
    dict(periodic=(True, True, True), world=3, walls=None, obstacles=False, kw={}),
    # two slabs that are each other's lower and upper neighbour; FP16-shifted storage
    dict(periodic=(False, True, True), world=2, walls=None, obstacles=False,
         kw=dict(storage="fp16")),
    # open z with wall faces on y and z, regularized obstacle surfaces cut by the slabs
    dict(periodic=(False, False, False), world=3, walls=(False, False, True, True, True, True),
         obstacles=True, kw={}),
    # local-strain relaxation, open z, uneven slab sizes
    dict(periodic=(True, False, False), world=4, walls=None, obstacles=False,
         kw=dict(grad_mode="local")),
])
def test_local_slabs_reproduce_the_undivided_domain_bit_for_bit(lib, case):
    from paper_1807_02284_gb300 import sharding
    sc = _scene(case["periodic"])
    steps = 7
    want = _undivided(sc, steps, case["walls"], case["obstacles"], **case["kw"])
    slabs = [_slab(sc, r, case["world"], case["walls"], case["obstacles"], **case["kw"])
             for r in range(case["world"])]
    sharding.step_local(slabs, steps)
    parts = [_owned(s) for s in slabs]
    for s in slabs:
        s.close()
    _assert_same(parts, want)


def test_plane_entry_point_checks(lib):
    import torch
    from paper_1807_02284_gb300 import lbm
    dom = lbm.Domain((8, 6, 5), 0.01, periodic=(True, True, True))
    assert dom.plane_bytes() == 8 * 6 * (27 * 4 + 17)   # population rows end 16-byte aligned
    buf = torch.zeros(dom.plane_bytes(), dtype=torch.uint8, device="cuda")
    for z in (-1, 5):
        with pytest.raises(lbm.LBMError) as ei:
            dom.pack_plane(z, buf)
        assert ei.value.status == lbm.LBM_ERR_INVALID_ARG
    with pytest.raises(lbm.LBMError) as ei:
        dom.pack_plane(0, buf, direction=2)
    assert ei.value.status == lbm.LBM_ERR_INVALID_ARG
    assert dom.plane_bytes(2) == 0
    sc = synth.random_scene(dims=(8, 6, 5), seed=3)
    dom.init_macro(f32(sc.blocks[0].u0), rho=f32(sc.blocks[0].rho0), c=f32(sc.blocks[0].c0))
    dom.step(2)
    f0 = dom.read_field(lbm.LBM_FIELD_F, lbm.LBM_F32).reshape(27, 5, 6, 8)
    dom.pack_plane(4, buf)
    dom.unpack_plane(0, buf)              # plane 0 now equals plane 4
    dom.sync()
    f = dom.read_field(lbm.LBM_FIELD_F, lbm.LBM_F32).reshape(27, 5, 6, 8)
    assert np.array_equal(f[:, 0], f[:, 4]) and not np.array_equal(f0[:, 0], f0[:, 4])
    from oracle import cmr
    cz = cmr.C[:, 2].numpy()              # fields are read in the paper's velocity order
    for direction in (+1, -1):
        slots = cz == direction
        nb = dom.plane_bytes(direction)
        assert nb == 9 * 48 * 4 + 48 * 17
        dom.pack_plane(3, buf[:nb], direction)
        dom.unpack_plane(1, buf[:nb], direction)
        dom.sync()
        g = dom.read_field(lbm.LBM_FIELD_F, lbm.LBM_F32).reshape(27, 5, 6, 8)
        assert np.array_equal(g[slots, 1], g[slots, 3])
        assert np.array_equal(g[~slots, 1], f[~slots, 1])    # the other slots are left alone
        f = g
    dom.close()
    ms = lbm.Domain((12, 12, 12), 0.01)
    ms.add_scale_block((2.0, 2.0, 2.0), 0.5, (8, 8, 8))
    buf = torch.zeros(ms.plane_bytes(), dtype=torch.uint8, device="cuda")
    with pytest.raises(lbm.LBMError) as ei:
        ms.pack_plane(0, buf)
    assert ei.value.status == lbm.LBM_ERR_UNSUPPORTED
    ms.close()
    half = lbm.Domain((5, 3, 4), 0.01, storage="fp16")
    assert half.plane_bytes() == 816 + 15 * 17        # 27 * 15 * 2 = 810 bytes, padded to 816
    with pytest.raises(ValueError):
        half.pack_plane(0, torch.zeros(half.plane_bytes() - 1, dtype=torch.uint8, device="cuda"))
    buf = torch.zeros(half.plane_bytes(), dtype=torch.uint8, device="cuda")
    half.pack_plane(3, buf)
    half.unpack_plane(1, buf)
    half.sync()
    for field in (lbm.LBM_FIELD_F, lbm.LBM_FIELD_U, lbm.LBM_FIELD_SCALAR):
        a = half.read_field(field, lbm.LBM_F32).reshape(-1, 4, 3, 5)
        assert np.array_equal(a[:, 1], a[:, 3])
    half.close()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _gloo_worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sc = _scene((False, True, True))
        s = _slab(sc, rank, world, None, False)
        s.step(6)                         # exchange through torch.distributed, then step
        q.put((rank, _owned(s)))
        s.close()
    finally:
        dist.barrier()
        dist.destroy_process_group()


def test_two_process_slabs_through_torch_distributed(lib):
    """Two processes, one slab each, on the same GPU: the exchange runs on the host (gloo,
    staged through host memory), so no kernel of one process waits for the other."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gloo_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    want = _undivided(_scene((False, True, True)), 6, None, False)
    _assert_same([r[1] for r in res], want)


def test_step_slab_argument_checks(lib):
    """lbm_step_slab refuses a missing or unaligned send buffer for a halo side, a slab with
    fewer than two owned planes, and domains with refined blocks."""
    import torch
    from paper_1807_02284_gb300 import lbm
    dom = lbm.Domain((8, 6, 6), 0.01, periodic=(True, True, False))
    nb = dom.plane_bytes(-1)
    buf = torch.zeros(nb + 16, dtype=torch.uint8, device="cuda")
    st = dom.lib.lbm_step_slab(dom.handle, 1, 0, None, None, None)
    assert st == lbm.LBM_ERR_INVALID_ARG
    st = dom.lib.lbm_step_slab(dom.handle, 1, 0, buf.data_ptr() + 8, None, None)
    assert st == lbm.LBM_ERR_INVALID_ARG                     # not 16-byte aligned
    dom.close()
    thin = lbm.Domain((8, 6, 3), 0.01, periodic=(True, True, False))
    b2 = torch.zeros(thin.plane_bytes(1), dtype=torch.uint8, device="cuda")
    st = thin.lib.lbm_step_slab(thin.handle, 1, 1, b2.data_ptr(), b2.data_ptr(), None)
    assert st == lbm.LBM_ERR_INVALID_ARG                     # one owned plane
    thin.close()
    multi = lbm.Domain((16, 16, 16), 0.01)
    multi.add_scale_block((4.0, 4.0, 4.0), 0.5, (8, 8, 8))
    st = multi.lib.lbm_step_slab(multi.handle, 0, 0, None, None, None)
    assert st == lbm.LBM_ERR_UNSUPPORTED
    multi.close()


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_slabs_on_the_two_node_kernel_reproduce_the_one_node_domain(lib, monkeypatch, storage):
    """The slab steps (send planes first, then the rest, as plane ranges) on the two-node
    kernel against the undivided domain on the one-node kernel, bit for bit."""
    from paper_1807_02284_gb300 import sharding
    sc = _scene((False, True, True))
    monkeypatch.setenv("LBM_TILE", "64,4,3")
    want = _undivided(sc, 7, None, False, storage=storage)
    monkeypatch.setenv("LBM_TILE", "64,4,20")
    slabs = [_slab(sc, r, 2, None, False, storage=storage) for r in range(2)]
    assert slabs[0].dom.info(0).nodes_per_thread == 2
    sharding.step_local(slabs, 7)
    parts = [_owned(s) for s in slabs]
    for s in slabs:
        s.close()
    _assert_same(parts, want)
