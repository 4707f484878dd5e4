"""Work placement across ranks (one process per GPU).

Independent simulations: batched simulations share nothing, so a multi-GPU run needs no
collective on the data path: each rank advances its own subset.  Subsets are chosen by
greedy largest-first bin packing on the lattice-node count, which keeps the slowest rank (the
one that sets the wall time) close to the mean.  Timing and throughput are combined with one
max / sum reduction.

One large domain (no counterpart in the paper, which runs one GPU): the domain is cut into
slabs of whole z-planes, one per rank.  Each slab is a domain of its own with one halo plane
on every side that borders another slab; before every step the edge planes of the current
state are exchanged point to point — the 9 populations (as stored) that cross the cut into
the receiving slab, velocity, scalar and node flags — so that every owned node sees the same
pull sources, lagged velocities and scalar samples as in the undivided domain.  One halo
plane is enough: the step reads only the 26 nearest neighbours and the scalar's departure
point moves at most one node per step.
"""
from __future__ import annotations

import heapq
from dataclasses import dataclass
from typing import List, Optional, Sequence, Tuple


def shard_by_cells(sizes: Sequence[int], world: int) -> List[List[int]]:
    """Indices of `sizes` per rank, largest first onto the least-loaded rank (ties -> lower
    rank).  Every index appears exactly once; each rank's list is sorted."""
    if world < 1:
        raise ValueError("world must be >= 1")
    heap = [(0, r) for r in range(world)]
    out: List[List[int]] = [[] for _ in range(world)]
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]), i))
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + int(sizes[i]), r))
    return [sorted(s) for s in out]


def rank_share(sizes: Sequence[int], rank: int, world: int) -> List[int]:
    return shard_by_cells(sizes, world)[rank]


def reduce_timing(seconds: float, work: float, group=None):
    """(max seconds over ranks, total work over ranks) with torch.distributed (any backend);
    with no process group the local values are returned."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return seconds, work
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([seconds], dtype=torch.float64, device=dev)
    w = torch.tensor([work], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(w, op=dist.ReduceOp.SUM, group=group)
    return float(t.item()), float(w.item())


# ----------------------------------------------------------------------- slabs along z

DOWN, UP = 0, 1     # message tags: a slab's first owned plane goes down, its last goes up
# Population direction carried by each message: a plane sent down fills the upper halo of
# the slab below, whose top nodes pull from it the populations with c_z = -1; a plane sent
# up carries those with c_z = +1.
DIRECTION = {DOWN: -1, UP: +1}


def slab_ranges(nz: int, world: int) -> List[Tuple[int, int]]:
    """Owned planes [z0, z1) per rank: nz split as evenly as possible, lower ranks first."""
    if world < 1 or nz < world:
        raise ValueError("need 1 <= world <= nz")
    base, extra = divmod(nz, world)
    out, z = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((z, z + n))
        z += n
    return out


@dataclass(frozen=True)
class SlabPlan:
    """One rank's slab: owned planes [z0, z1) of nz, halo planes below (lo) and above (hi),
    the neighbouring ranks and the local domain's z periodicity."""
    rank: int
    world: int
    nz: int
    z0: int
    z1: int
    lo: int
    hi: int
    lower: Optional[int]
    upper: Optional[int]
    local_periodic_z: bool

    @property
    def local_nz(self) -> int:
        return self.z1 - self.z0 + self.lo + self.hi

    @property
    def owned(self) -> slice:
        """Local z indices of the owned planes."""
        return slice(self.lo, self.lo + self.z1 - self.z0)

    def global_planes(self) -> List[int]:
        """Global z index of every local plane (halo planes included)."""
        return [(self.z0 - self.lo + i) % self.nz for i in range(self.local_nz)]

    def transfers(self):
        """The halo exchange of one step, in issue order: (kind, local z, peer rank, tag).
        Sends come first, then receives; between one pair of ranks the messages of each
        direction are matched in this order, which also holds for two ranks that are each
        other's lower and upper neighbour."""
        out = []
        if self.lower is not None:
            out.append(("send", self.lo, self.lower, DOWN))
        if self.upper is not None:
            out.append(("send", self.lo + self.z1 - self.z0 - 1, self.upper, UP))
        if self.upper is not None:
            out.append(("recv", self.local_nz - 1, self.upper, DOWN))
        if self.lower is not None:
            out.append(("recv", 0, self.lower, UP))
        return out


def slab_plan(nz: int, world: int, rank: int, periodic_z: bool) -> SlabPlan:
    """The slab of `rank`: with a periodic z axis every slab has both halos (a single slab
    keeps its own periodic wrap and has none); otherwise the global end faces stay the end
    faces of the first and last slab, without a halo there."""
    z0, z1 = slab_ranges(nz, world)[rank]
    if world == 1:
        return SlabPlan(rank, 1, nz, z0, z1, 0, 0, None, None, bool(periodic_z))
    lower = (rank - 1) % world if (periodic_z or rank > 0) else None
    upper = (rank + 1) % world if (periodic_z or rank < world - 1) else None
    return SlabPlan(rank, world, nz, z0, z1, int(lower is not None), int(upper is not None),
                    lower, upper, False)


class SlabDomain:
    """One rank's slab of a domain of `dims` (nx, ny, nz) cut along z.

    Global inputs (flags, walls, inflow records, initial fields) are given for the whole
    domain and sliced here; ``read_owned`` returns this slab's owned planes.  ``step`` runs
    the halo exchange through ``torch.distributed`` before every step; ``step_local``
    advances several slabs held by one process.  ``make_domain(dims, periodic)`` builds the
    slab's domain (default: an ``lbm.Domain`` with the remaining keyword arguments)."""

    def __init__(self, dims, nu, rank=0, world=1, periodic=(False, False, False),
                 make_domain=None, **domain_kw):
        import torch
        nx, ny, nz = (int(v) for v in dims)
        self.dims = (nx, ny, nz)
        self.periodic = tuple(bool(p) for p in periodic)
        self.plan = slab_plan(nz, world, rank, self.periodic[2])
        local_periodic = (self.periodic[0], self.periodic[1], self.plan.local_periodic_z)
        if make_domain is None:
            from . import lbm

            def make_domain(d, p):
                return lbm.Domain(d, nu, periodic=p, **domain_kw)
        self.dom = make_domain((nx, ny, self.plan.local_nz), local_periodic)
        dev = getattr(self.dom, "plane_device", "cuda")
        self.bufs = {(k, tag): torch.empty(self.dom.plane_bytes(DIRECTION[tag]),
                                           dtype=torch.uint8, device=dev)
                     for (k, _, _, tag) in self.plan.transfers()}
        # the halos hold the neighbours' current edge planes (an exchange or a pipelined step
        # since the state last changed from outside)
        self._halos_current = False
        self._pack_stream = None

    # ------------------------------------------------------------------ global inputs
    def local(self, a):
        """Local planes (halos included) of a global array shaped (..., nz, ny, nx)."""
        import numpy as np
        return np.ascontiguousarray(np.take(np.asarray(a), self.plan.global_planes(), axis=-3))

    def owned(self, a):
        """Owned planes of a local array shaped (..., local_nz, ny, nx)."""
        return a[..., self.plan.owned, :, :]

    def set_flags(self, flags):
        self.dom.set_flags(self.local(flags))
        self._halos_current = False

    def set_walls(self, faces, obstacles=False):
        """Wall faces (x-, x+, y-, y+, z-, z+) of the whole domain: a z face belongs to the
        slab that holds that end of the (non-periodic) z axis."""
        faces = [bool(f) for f in faces]
        if (faces[4] or faces[5]) and self.periodic[2]:
            raise ValueError("z wall faces need a non-periodic z axis")
        faces[4] = faces[4] and self.plan.lo == 0 and self.plan.z0 == 0
        faces[5] = faces[5] and self.plan.hi == 0 and self.plan.z1 == self.plan.nz
        self.dom.set_walls(faces, obstacles=obstacles)
        self._halos_current = False

    def set_inflow(self, records):
        """Inflow records in global coordinates; those on a local plane are kept, moved to
        local z (a record on a halo plane also arrives with the owner's flags)."""
        import numpy as np
        from . import lbm
        rec = np.asarray(records, dtype=lbm.INFLOW_RECORD)
        planes = np.asarray(self.plan.global_planes())
        keep = []
        for i, g in enumerate(planes):
            r = rec[rec["z"] == g].copy()
            r["z"] = i
            keep.append(r)
        out = np.concatenate(keep) if keep else rec[:0]
        if len(out):
            self.dom.set_inflow(out)
        self._halos_current = False

    def init_macro(self, u, rho=None, c=None):
        import numpy as np
        loc = [None if a is None else self.local(np.asarray(a, dtype=np.float32))
               for a in (u, rho, c)]
        self.dom.init_macro(loc[0], rho=loc[1], c=loc[2])
        self._halos_current = False

    def read_owned(self, field, dtype=None):
        """A field of this slab's owned planes, shaped (comp, planes, ny, nx) or
        (planes, ny, nx) for one-component fields."""
        from . import lbm
        dt = lbm.LBM_F64 if dtype is None else dtype
        a = self.dom.read_field(field, dt)
        nx, ny, _ = self.dims
        comp = a.size // (nx * ny * self.plan.local_nz)
        a = a.reshape((comp, self.plan.local_nz, ny, nx))
        a = self.owned(a)
        return a[0] if comp == 1 else a

    def gather_owned(self, field, dtype=None, dst=0, group=None):
        """A field of the whole domain, assembled on rank `dst` from every rank's owned
        planes (read back to the host, sent with ``gather_object``); other ranks get None.
        Without a process group the slab's own planes are returned."""
        import numpy as np
        import torch.distributed as dist
        a = self.read_owned(field, dtype)
        if not (dist.is_available() and dist.is_initialized()):
            return a
        me = dist.get_rank(group)
        parts = [None] * dist.get_world_size(group) if me == dst else None
        g_dst = dst if group is None else dist.get_global_rank(group, dst)
        dist.gather_object((self.plan.z0, a), parts, dst=g_dst, group=group)
        if me != dst:
            return None
        parts.sort(key=lambda p: p[0])
        return np.concatenate([p[1] for p in parts], axis=-3)

    # ------------------------------------------------------------------ halo exchange
    def _pack(self):
        for kind, z, _, tag in self.plan.transfers():
            if kind == "send":
                self.dom.pack_plane(z, self.bufs[(kind, tag)], DIRECTION[tag])

    def _unpack(self, source=None):
        for kind, z, peer, tag in self.plan.transfers():
            if kind == "recv":
                buf = self.bufs[(kind, tag)] if source is None else source(peer, tag)
                self.dom.unpack_plane(z, buf, DIRECTION[tag])

    def exchange(self, group=None):
        """Halo exchange of the current state with the neighbouring ranks (any backend;
        device buffers are staged through host memory for backends other than NCCL)."""
        tr = self.plan.transfers()
        if not tr:
            return
        self._pack()
        self.dom.sync()
        self._transport(group)
        self._unpack()
        self._halos_current = True

    def _transport(self, group=None, stream=None):
        """Sends the packed edge planes and receives the neighbours' into the recv buffers.
        With NCCL and a `stream` (the stream the planes were packed on) nothing waits on the
        host: the messages follow the packing, and the domain's stream waits for them."""
        import torch
        import torch.distributed as dist
        tr = self.plan.transfers()
        nccl = dist.get_backend(group) == "nccl"
        if stream is not None and nccl:
            ops = []
            for kind, _, peer, tag in tr:
                g_peer = peer if group is None else dist.get_global_rank(group, peer)
                fn = dist.isend if kind == "send" else dist.irecv
                ops.append(dist.P2POp(fn, self.bufs[(kind, tag)], g_peer, group, tag))
            with torch.cuda.stream(stream):
                reqs = dist.batch_isend_irecv(ops)
            with torch.cuda.stream(self.dom.torch_stream):
                for req in reqs:
                    req.wait()
            return
        if stream is not None:
            stream.synchronize()
        staged = {}
        ops = []
        for kind, _, peer, tag in tr:
            t = self.bufs[(kind, tag)]
            if t.is_cuda and not nccl:
                t = staged.setdefault((kind, tag), t.cpu())
            g_peer = peer if group is None else dist.get_global_rank(group, peer)
            fn = dist.isend if kind == "send" else dist.irecv
            ops.append(dist.P2POp(fn, t, g_peer, group, tag))
        for req in dist.batch_isend_irecv(ops):
            req.wait()
        for (kind, tag), t in staged.items():
            if kind == "recv":
                self.bufs[(kind, tag)].copy_(t)
        if any(t.is_cuda for t in self.bufs.values()):
            torch.cuda.synchronize()

    def _step_sends(self, stream=None):
        """One step of this slab whose new edge planes are packed into the send buffers on
        `stream` while its other planes step (the domain's lbm_step_slab)."""
        lo, hi = self.plan.lower is not None, self.plan.upper is not None
        self.dom.step_slab(lo, hi, self.bufs.get(("send", DOWN)), self.bufs.get(("send", UP)),
                           stream)

    def step(self, n=1, group=None):
        """n steps of the whole domain, this rank's slab.  With a domain that has
        ``step_slab``: an exchange of the current edge planes if the halos are not current,
        then per step the send planes first, their transport while the other planes step,
        and the unpack into the halos before the next step.  Otherwise: exchange, then step."""
        if not self.plan.transfers():
            self.dom.step(int(n))
            return
        if not hasattr(self.dom, "step_slab"):
            for _ in range(int(n)):
                self.exchange(group)
                self.dom.step(1)
            self._halos_current = False
            return
        import torch
        if not self._halos_current:
            self.exchange(group)
        on_gpu = any(t.is_cuda for t in self.bufs.values())
        if on_gpu and self._pack_stream is None:
            self._pack_stream = torch.cuda.Stream(device=next(iter(self.bufs.values())).device)
        for _ in range(int(n)):
            self._step_sends(self._pack_stream)
            self._transport(group, self._pack_stream if on_gpu else None)
            self._unpack()
        self._halos_current = True

    def sync(self):
        self.dom.sync()

    def close(self):
        self.dom.close()


def step_local(slabs: Sequence[SlabDomain], n: int = 1):
    """n steps of a domain whose slabs (rank = list index) are all held by this process.
    With domains that have ``step_slab``: the current edge planes are exchanged once if the
    halos are not current, then per step every slab steps its send planes first and packs
    them on one shared stream while its other planes step, and every neighbour unpacks them
    from the sender's buffer once that stream has packed them.  Otherwise every slab packs
    its edge planes, every neighbour unpacks them, then every slab steps.  Slabs on one
    stream are ordered by it (nothing waits on the host); otherwise each phase waits for the
    previous one on every slab's stream."""
    by_rank = {s.plan.rank: s for s in slabs}
    if sorted(by_rank) != list(range(len(slabs))):
        raise ValueError("slabs must be ranks 0 .. n-1 of one cut")
    s0 = getattr(slabs[0].dom, "torch_stream", None)
    shared = s0 is not None and all(getattr(s.dom, "torch_stream", None) == s0 for s in slabs)

    def sender(peer, tag):
        return by_rank[peer].bufs[("send", tag)]

    def wait_all():
        if not shared:
            for s in slabs:
                s.sync()

    def exchange_all():
        for s in slabs:
            s._pack()
        wait_all()
        for s in slabs:
            s._unpack(sender)
        wait_all()
    if len(slabs) > 1 and all(hasattr(s.dom, "step_slab") for s in slabs):
        import torch
        if not all(s._halos_current for s in slabs):
            exchange_all()
        on_gpu = any(t.is_cuda for s in slabs for t in s.bufs.values())
        pack = None
        if on_gpu:
            if slabs[0]._pack_stream is None:
                slabs[0]._pack_stream = torch.cuda.Stream(
                    device=next(iter(slabs[0].bufs.values())).device)
            pack = slabs[0]._pack_stream
        for _ in range(int(n)):
            for s in slabs:
                s._step_sends(pack)
            if on_gpu:
                done = pack.record_event()
                for s in slabs:
                    s.dom.torch_stream.wait_event(done)
            wait_all()
            for s in slabs:
                s._unpack(sender)
            wait_all()
        for s in slabs:
            s._halos_current = True
        return
    for _ in range(int(n)):
        exchange_all()
        for s in slabs:
            s.dom.step(1)
        wait_all()
    for s in slabs:
        s._halos_current = False


# ------------------------------------------------ blocks of one continuous-scale domain

# One reference step of Algorithm 1 reads, for every refined block, its prior-mapping source
# around the block's scale boundary at t_n and at t_n + dt_0, and writes its post-mapping
# into every coarser block.  With the blocks of one domain placed on several ranks, every
# rank holds the whole domain and steps it phase by phase (lbm_step_phase), computing the
# phases of the blocks it owns; the node boxes those mappings touch move between phases:
#   ("prior", b) before block b's sub-cycle: the source block's boxes at t_n (LEVEL_START,
#                with the source's own scale boundary at t_n refreshed by its sub-cycle) and
#                at t_n + dt_0 (LEVEL_CURRENT, after every earlier block's post-mapping into
#                it), to b's owner;
#   ("post", b)  after block b's post-mapping, computed by b's owner into its copy of every
#                coarser block: the written box to that block's owner (obstacle and
#                scale-boundary nodes of the box are left alone there: no mapping writes
#                them).
SOLID_BIT, GHOST_BIT = 1, 8


@dataclass(frozen=True)
class BoxMove:
    """One node box moved between ranks at one stage of a reference step."""
    stage: tuple
    block: int
    level: int
    lo: tuple
    hi: tuple
    src: int
    dst: int
    skip: int


def place_blocks(updates: Sequence[int], world: int) -> List[int]:
    """Owner rank of every block: largest-first packing of the lattice updates per reference
    step (nodes x sub-steps), as for independent simulations."""
    owner = [0] * len(updates)
    for r, idx in enumerate(shard_by_cells(updates, world)):
        for i in idx:
            owner[i] = r
    return owner


def block_moves(parents: Sequence[int], owner: Sequence[int], boxes) -> List[BoxMove]:
    """The box moves of one reference step, in stage order.  parents[b] is block b's
    prior-mapping source (-1: not a refined block); boxes(b, kind, other) lists the (lo, hi)
    boxes of lbm_mapping_boxes."""
    from . import lbm
    refined = [b for b in range(len(parents)) if parents[b] >= 0]
    moves: List[BoxMove] = []
    for b in refined:
        p = parents[b]
        if owner[p] != owner[b]:
            for level in (lbm.LBM_LEVEL_START, lbm.LBM_LEVEL_CURRENT):
                for lo, hi in boxes(b, lbm.LBM_BOX_PRIOR_SOURCE, p):
                    moves.append(BoxMove(("prior", b), p, level, tuple(lo), tuple(hi),
                                         owner[p], owner[b], 0))
        for k in range(len(parents)):
            if k == b or owner[k] == owner[b]:
                continue
            for lo, hi in boxes(b, lbm.LBM_BOX_POST_TARGET, k):
                moves.append(BoxMove(("post", b), k, lbm.LBM_LEVEL_CURRENT, tuple(lo), tuple(hi),
                                     owner[b], owner[k], SOLID_BIT | GHOST_BIT))
    return moves


class PlacedDomain:
    """One rank's view of a continuous-scale domain whose blocks are placed on ranks.

    ``dom`` holds the whole domain (every block built, flagged and initialised the same way
    on every rank); ``owner[b]`` is the rank that computes block b.  ``step`` advances one
    reference step through ``torch.distributed`` point-to-point messages (any backend;
    device buffers are staged through host memory for backends other than NCCL);
    ``step_local`` advances the ranks held by one process."""

    def __init__(self, dom, owner: Sequence[int], rank: int):
        import torch
        from . import lbm
        self.dom = dom
        self.rank = int(rank)
        nb = dom.n_blocks()
        self.owner = [int(o) for o in owner]
        if len(self.owner) != nb:
            raise ValueError("one owner per block")
        self.parents = [dom.info(b).parent for b in range(nb)]
        self.refined = [b for b in range(nb) if self.parents[b] >= 0]
        self.moves = block_moves(self.parents, self.owner,
                                 lambda b, kind, other: dom.mapping_boxes(b, kind, other))
        dev = getattr(dom, "box_device", "cuda")
        self.bufs = {}
        for i, m in enumerate(self.moves):
            if self.rank in (m.src, m.dst):
                nbytes = dom.box_bytes(m.block, m.lo, m.hi)
                self.bufs[i] = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        self.lbm = lbm

    def stage_moves(self, stage):
        return [(i, m) for i, m in enumerate(self.moves) if m.stage == stage]

    def pack(self, stage):
        for i, m in self.stage_moves(stage):
            if m.src == self.rank:
                self.dom.pack_box(m.block, m.level, m.lo, m.hi, self.bufs[i])

    def unpack(self, stage, source=None):
        for i, m in self.stage_moves(stage):
            if m.dst == self.rank:
                buf = self.bufs[i] if source is None else source(i, m)
                self.dom.unpack_box(m.block, m.level, m.lo, m.hi, buf, m.skip)

    def exchange(self, stage, group=None):
        """The moves of one stage through torch.distributed (tag = move index)."""
        mine = [(i, m) for i, m in self.stage_moves(stage) if self.rank in (m.src, m.dst)]
        if not mine:
            return
        import torch
        import torch.distributed as dist
        self.pack(stage)
        self.dom.sync()
        nccl = dist.get_backend(group) == "nccl"
        staged, ops = {}, []
        for i, m in mine:
            t = self.bufs[i]
            if t.is_cuda and not nccl:
                t = staged.setdefault(i, t.cpu())
            peer = m.dst if m.src == self.rank else m.src
            g_peer = peer if group is None else dist.get_global_rank(group, peer)
            fn = dist.isend if m.src == self.rank else dist.irecv
            ops.append(dist.P2POp(fn, t, g_peer, group, i))
        for req in dist.batch_isend_irecv(ops):
            req.wait()
        for i, t in staged.items():
            if self.moves[i].dst == self.rank:
                self.bufs[i].copy_(t)
        if any(t.is_cuda for t in self.bufs.values()):
            torch.cuda.synchronize()
        self.unpack(stage)

    def schedule(self):
        """One reference step as a list of ("phase", phase, block) and ("stage", stage)
        items, in order."""
        lbm = self.lbm
        items = [("phase", lbm.LBM_PHASE_BEGIN, 0), ("phase", lbm.LBM_PHASE_REFERENCE, 0)]
        for b in self.refined:
            items += [("stage", ("prior", b)), ("phase", lbm.LBM_PHASE_BLOCK, b),
                      ("phase", lbm.LBM_PHASE_POST, b), ("stage", ("post", b))]
        items.append(("phase", lbm.LBM_PHASE_END, 0))
        return items

    def run_phase(self, phase, block):
        """One phase, computed if this rank owns the block it advances."""
        lbm = self.lbm
        compute = phase in (lbm.LBM_PHASE_REFERENCE, lbm.LBM_PHASE_BLOCK, lbm.LBM_PHASE_POST) \
            and self.owner[block] == self.rank
        self.dom.step_phase(phase, block, compute)

    def step(self, n=1, group=None):
        """n reference steps, exchanging through torch.distributed."""
        for _ in range(int(n)):
            for item in self.schedule():
                if item[0] == "phase":
                    self.run_phase(item[1], item[2])
                else:
                    self.exchange(item[1], group)

    def sync(self):
        self.dom.sync()


def step_placed_local(ranks: Sequence[PlacedDomain], n: int = 1):
    """n reference steps of a domain whose ranks (list index = rank) are all held by this
    process, in lockstep: every rank runs each phase, and at every stage each sender packs
    its boxes and each receiver unpacks them from the sender's buffer.  With every rank's
    domain on one stream nothing waits on the host; otherwise each stage waits for every
    rank's stream."""
    if [r.rank for r in ranks] != list(range(len(ranks))):
        raise ValueError("ranks must be 0 .. n-1 of one placement")
    s0 = getattr(ranks[0].dom, "torch_stream", None)
    shared = s0 is not None and all(getattr(r.dom, "torch_stream", None) == s0 for r in ranks)

    def wait_all():
        if not shared:
            for r in ranks:
                r.dom.sync()

    def source(i, m):
        return ranks[m.src].bufs[i]

    for _ in range(int(n)):
        for item in ranks[0].schedule():
            if item[0] == "phase":
                for r in ranks:
                    r.run_phase(item[1], item[2])
            else:
                wait_all()
                for r in ranks:
                    r.pack(item[1])
                wait_all()
                for r in ranks:
                    r.unpack(item[1], source)
