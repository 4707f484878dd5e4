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


# ------------------------------------------------------------------ slabs of one domain

class _StencilDomain:
    """Host stand-in for a slab's domain with the library's data dependence, in integers so
    that an exchange mistake (a wrong plane, peer, slot or direction) changes owned values
    exactly: slot s of `a` moves along z by c_z = s - 1 and is pulled from x - c_z with the
    library's neighbour rule (periodic axes wrap, open axes clamp) and from all 9 x/y
    neighbours; `g` (like the lagged velocity) enters through central differences along z.
    A plane of direction +1 / -1 carries slot 2 / 0 and g, direction 0 all slots.  Plane
    buffers live on the host."""
    plane_device = "cpu"
    P = 1_000_003

    def __init__(self, dims, periodic):
        self.nx, self.ny, self.nz = dims
        self.periodic = periodic
        self.a = np.zeros((3, self.nz, self.ny, self.nx), np.int64)
        self.g = np.zeros((self.nz, self.ny, self.nx), np.int64)

    @staticmethod
    def slots(direction):
        return {1: [2], -1: [0], 0: [0, 1, 2]}[direction]

    def plane_bytes(self, direction=0):
        return (len(self.slots(direction)) + 1) * self.nx * self.ny * 8

    def pack_plane(self, z, buf, direction=0):
        rows = [self.a[s, z] for s in self.slots(direction)] + [self.g[z]]
        buf.numpy()[:] = np.stack(rows).reshape(-1).view(np.uint8)

    def unpack_plane(self, z, buf, direction=0):
        rows = buf.numpy().view(np.int64).reshape(-1, self.ny, self.nx)
        for r, s in enumerate(self.slots(direction)):
            self.a[s, z] = rows[r]
        self.g[z] = rows[-1]

    def sync(self):
        pass

    def step_slab(self, lo, hi, send_lo=None, send_hi=None, pack_stream=None):
        """The library's slab step: a step, then the new first / last owned planes packed
        (direction -1 / +1); the halo planes are left as stale as the library leaves them."""
        keep_a, keep_g = self.a.copy(), self.g.copy()
        self.step(1)
        for z, on in ((0, lo), (self.nz - 1, hi)):
            if on:
                self.a[:, z] = keep_a[:, z] - 1          # stale, and visibly so
                self.g[z] = keep_g[z] - 1
        if lo:
            self.pack_plane(1, send_lo, -1)
        if hi:
            self.pack_plane(self.nz - 2, send_hi, +1)

    def read_field(self, field, dtype=None):
        return self.a.reshape(-1).copy()

    def _nbr(self, ax, o):
        m = (self.nz, self.ny, self.nx)[ax]
        j = np.arange(m) + o
        return j % m if self.periodic[2 - ax] else np.clip(j, 0, m - 1)

    def step(self, n=1):
        for _ in range(n):
            pulled = np.zeros_like(self.a)
            for s in range(3):
                zs = self._nbr(0, -(s - 1))
                for k, (dy, dx) in enumerate(np.ndindex(3, 3)):
                    ys, xs = self._nbr(1, dy - 1), self._nbr(2, dx - 1)
                    pulled[s] += (k + 1 + 3 * s) * self.a[s][np.ix_(zs, ys, xs)]
            dg = self.g[self._nbr(0, 1)] - self.g[self._nbr(0, -1)]
            mix = np.array([[2, 1, 0], [1, 3, 1], [0, 1, 5]])
            self.a = (np.einsum("st,tzyx->szyx", mix, pulled) + dg) % self.P
            self.g = (pulled.sum(0) + 7 * self.g) % self.P


def _stencil_init(shape_zyx, seed):
    rng = np.random.default_rng(seed)
    return (rng.integers(0, 1000, size=(3,) + shape_zyx).astype(np.int64),
            rng.integers(0, 1000, size=shape_zyx).astype(np.int64))


def _stencil_reference(a, g, periodic, steps):
    d = _StencilDomain(g.shape[::-1], periodic)
    d.a, d.g = a.copy(), g.copy()
    d.step(steps)
    return d.a, d.g


class _PlainStencilDomain(_StencilDomain):
    """The stand-in without a slab step: exchange, then a plain step of every plane."""
    @property
    def step_slab(self):
        raise AttributeError("step_slab")


def _stencil_slabs(a, g, periodic, world, ranks, plain=False):
    out = []
    for r in ranks:
        s = sharding.SlabDomain(g.shape[::-1], 0.0, rank=r, world=world, periodic=periodic,
                                make_domain=_PlainStencilDomain if plain else _StencilDomain)
        s.dom.a, s.dom.g = s.local(a), s.local(g)
        out.append(s)
    return out


def _owned_stencil(slabs):
    return (np.concatenate([s.owned(s.dom.a) for s in slabs], axis=1),
            np.concatenate([s.owned(s.dom.g) for s in slabs], axis=0))


def test_slab_plan_covers_every_plane_once_with_the_right_halos():
    for nz in (5, 7, 16):
        for world in (1, 2, 3, 5):
            for per in (False, True):
                plans = [sharding.slab_plan(nz, world, r, per) for r in range(world)]
                owned = [g for p in plans for g in p.global_planes()[p.owned]]
                assert owned == list(range(nz))
                for p in plans:
                    g = p.global_planes()
                    if p.lo:
                        assert g[0] == (p.z0 - 1) % nz
                    if p.hi:
                        assert g[-1] == p.z1 % nz
                    assert (p.lo == 0) == (world == 1 or (not per and p.rank == 0))
                    assert (p.hi == 0) == (world == 1 or (not per and p.rank == world - 1))
                    assert p.local_periodic_z == (per and world == 1)
                # every send is one receive of the peer, of the same global plane
                for p in plans:
                    for kind, z, peer, tag in p.transfers():
                        if kind != "send":
                            continue
                        q = plans[peer]
                        rz = [zz for k2, zz, pr, t2 in q.transfers()
                              if k2 == "recv" and pr == p.rank and t2 == tag]
                        assert len(rz) == 1
                        assert q.global_planes()[rz[0]] == p.global_planes()[z]
    with pytest.raises(ValueError):
        sharding.slab_ranges(3, 4)


@pytest.mark.parametrize("plain", [False, True])
@pytest.mark.parametrize("world", [1, 2, 3])
@pytest.mark.parametrize("periodic", [(True, False, True), (False, True, False)])
def test_local_slabs_reproduce_the_undivided_stencil(world, periodic, plain):
    """Slabs of one process: the pipelined slab step (send planes first, halo planes left
    stale until the unpack) and, with plain=True, exchange-then-step; stepped in two calls
    (the pipelined path keeps its halos current between them)."""
    a, g = _stencil_init((9, 5, 6), 7)
    want = _stencil_reference(a, g, periodic, 4)
    slabs = _stencil_slabs(a, g, periodic, world, range(world), plain)
    sharding.step_local(slabs, 3)
    sharding.step_local(slabs, 1)
    got = _owned_stencil(slabs)
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
    if world > 1:
        # without the exchange, or with the two directions swapped, the owned planes next
        # to a cut go wrong
        slabs = _stencil_slabs(a, g, periodic, world, range(world))
        for s in slabs:
            s.dom.step(4)
        assert not np.array_equal(_owned_stencil(slabs)[0], want[0])
        swapped = {sharding.DOWN: +1, sharding.UP: -1}
        old = dict(sharding.DIRECTION)
        try:
            sharding.DIRECTION.update(swapped)
            slabs = _stencil_slabs(a, g, periodic, world, range(world))
            sharding.step_local(slabs, 4)
        finally:
            sharding.DIRECTION.update(old)
        assert not np.array_equal(_owned_stencil(slabs)[0], want[0])


def _slab_worker(rank, world, port, periodic, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    a, g = _stencil_init((8, 4, 5), 11)
    (s,) = _stencil_slabs(a, g, periodic, world, [rank])
    s.step(3)
    whole = s.gather_owned(0, dst=world - 1)           # field argument unused by the stand-in
    q.put((rank, s.owned(s.dom.a), s.owned(s.dom.g), whole))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,periodic", [(2, (False, False, True)), (2, (True, True, False)),
                                            (3, (False, True, True))])
def test_gloo_slab_exchange_reproduces_the_undivided_stencil(world, periodic):
    """Two ranks that are each other's lower and upper neighbour (periodic z), a plain cut
    (open z) and a ring of three: the exchange goes through torch.distributed
    point-to-point messages."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_slab_worker, args=(r, world, port, periodic, q))
             for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=120) for _ in procs), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    a, g = _stencil_init((8, 4, 5), 11)
    want = _stencil_reference(a, g, periodic, 3)
    assert np.array_equal(np.concatenate([r[1] for r in res], axis=1), want[0])
    assert np.array_equal(np.concatenate([r[2] for r in res], axis=0), want[1])
    assert all(r[3] is None for r in res[:-1])         # assembled on the last rank only
    assert np.array_equal(res[-1][3], want[0])


class _RecordingDomain:
    """Records what a slab hands to its domain (flags, walls, inflow records, fields)."""
    plane_device = "cpu"

    def __init__(self, dims, periodic):
        self.dims, self.periodic, self.calls = dims, periodic, {}

    def plane_bytes(self, direction=0):
        return 16

    def set_flags(self, flags):
        self.calls["flags"] = flags

    def set_walls(self, faces, obstacles=False):
        self.calls["walls"] = (list(faces), obstacles)

    def set_inflow(self, records):
        self.calls["inflow"] = records

    def init_macro(self, u, rho=None, c=None):
        self.calls["init"] = (u, rho, c)


def test_slab_inputs_are_sliced_from_the_global_domain():
    from paper_1807_02284_gb300 import lbm
    nx, ny, nz = 4, 3, 10
    flags = np.arange(nz * ny * nx, dtype=np.int64).reshape(nz, ny, nx) % 251
    u = np.random.default_rng(2).random((3, nz, ny, nx))
    rec = np.zeros(4, dtype=lbm.INFLOW_RECORD)
    rec["z"] = [0, 3, 4, 9]
    rec["x"] = [1, 2, 3, 0]
    for per in (False, True):
        slabs = [sharding.SlabDomain((nx, ny, nz), 0.0, rank=r, world=3,
                                     periodic=(False, False, per), make_domain=_RecordingDomain)
                 for r in range(3)]
        for s in slabs:
            s.set_flags(flags.astype(np.uint8))
            s.set_walls((True, False, False, True, not per, not per), obstacles=True)
            s.set_inflow(rec)
            s.init_macro(u, c=u[0])
            g = s.plan.global_planes()
            d = s.dom
            assert d.dims == (nx, ny, len(g)) and d.periodic == (False, False, False)
            assert np.array_equal(d.calls["flags"], flags[g].astype(np.uint8))
            assert np.array_equal(d.calls["init"][0], u[:, g].astype(np.float32))
            assert d.calls["init"][1] is None
            assert np.array_equal(d.calls["init"][2], u[0][g].astype(np.float32))
            faces, obst = d.calls["walls"]
            assert faces[:4] == [True, False, False, True] and obst
            # a z wall face only where the slab holds that end of the open axis
            assert faces[4] == (not per and s.plan.rank == 0)
            assert faces[5] == (not per and s.plan.rank == 2)
            r = d.calls["inflow"]
            want = sorted((int(x), g.index(int(z))) for x, z in zip(rec["x"], rec["z"])
                          if int(z) in g)
            assert sorted(zip(r["x"].tolist(), r["z"].tolist())) == want
    with pytest.raises(ValueError):
        sharding.SlabDomain((nx, ny, nz), 0.0, rank=0, world=2, periodic=(False, False, True),
                            make_domain=_RecordingDomain).set_walls((False,) * 4 + (True, False))
