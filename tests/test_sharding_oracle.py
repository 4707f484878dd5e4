"""The slab cut of one domain (one halo plane per cut; per step the 9 populations that cross
the cut into the receiving slab, the velocity, the scalar and the flags) reproduces the
undivided domain under the FP64 oracle's step, on CPU: the exchange carries everything an
owned node reads (pull sources, bounce-back sources, lagged central differences, the
scalar's departure point).  Obstacles here take halfway bounce-back; the regularized
obstacle surface, whose halo status the library ships in the flags, is covered by the
GPU test of the cut."""
import dataclasses

import numpy as np
import pytest
import torch

import synth
from oracle import cmr, grid
from paper_1807_02284_gb300 import sharding
from tests.helpers import f32

CZ = cmr.C[:, 2].numpy()


class _OracleSlab:
    """A slab's domain advanced by the oracle; planes hold float64 rows (populations in the
    oracle's order, selected by c_z, then u, c and the flags)."""
    plane_device = "cpu"

    def __init__(self, dims, periodic, params):
        self.dims = dims
        self.p = dataclasses.replace(params, periodic=tuple(periodic))
        self.flags = None
        self.st = None

    @staticmethod
    def _slots(direction):
        return np.nonzero(CZ == direction)[0] if direction else np.arange(27)

    def plane_bytes(self, direction=0):
        nx, ny, _ = self.dims
        return (len(self._slots(direction)) + 5) * nx * ny * 8

    def set_flags(self, flags):
        self.flags = np.asarray(flags, np.uint8)

    def set_walls(self, faces, obstacles=False):
        self.p = dataclasses.replace(self.p, walls=tuple(bool(f) for f in faces),
                                     obstacle_walls=bool(obstacles))

    def init_macro(self, u, rho=None, c=None):
        self.st = grid.init_state(np.asarray(rho, np.float64), np.asarray(u, np.float64),
                                  np.asarray(c, np.float64), self.flags)

    def pack_plane(self, z, buf, direction=0):
        st = self.st
        rows = [st.f[q, z].numpy() for q in self._slots(direction)]
        rows += [st.u[a, z].numpy() for a in range(3)] + [st.c[z].numpy(),
                                                          st.flags[z].numpy().astype(np.float64)]
        buf.numpy()[:] = np.stack(rows).reshape(-1).view(np.uint8)

    def unpack_plane(self, z, buf, direction=0):
        nx, ny, _ = self.dims
        rows = torch.as_tensor(buf.numpy().view(np.float64).reshape(-1, ny, nx).copy())
        for r, q in enumerate(self._slots(direction)):
            self.st.f[q, z] = rows[r]
        k = len(self._slots(direction))
        self.st.u[:, z] = rows[k:k + 3]
        self.st.c[z] = rows[k + 3]
        self.st.flags[z] = rows[k + 4].to(torch.uint8)

    def step(self, n=1):
        for _ in range(n):
            self.st = grid.step(self.st, self.p)

    def sync(self):
        pass


def _scene(periodic):
    sc = synth.random_scene(dims=(9, 8, 12), seed=17, periodic=periodic, nu=0.004,
                            spheres=[(4.0, 4.0, 4.0, 2.2), (5.0, 3.5, 8.0, 2.0)],
                            inflow=(4, 6, 2.0, 0.06))
    sc.blocks[0].flags[5:7, 1:3, 5:7] |= synth.SCALAR_SRC
    return sc


def _run(case, steps=3):
    sc = _scene(case["periodic"])
    b = sc.blocks[0]
    params = grid.Params(nu=sc.nu, periodic=sc.periodic, adaptive=sc.adaptive,
                         c_src=sc.c_src, grad_mode=case["grad"])
    full = _OracleSlab(b.dims, sc.periodic, params)
    full.set_flags(b.flags)
    if case["walls"]:
        full.set_walls(case["walls"])
    full.init_macro(f32(b.u0), rho=f32(b.rho0), c=f32(b.c0))
    full.step(steps)

    slabs = [sharding.SlabDomain(b.dims, sc.nu, rank=r, world=case["world"],
                                 periodic=sc.periodic,
                                 make_domain=lambda d, p: _OracleSlab(d, p, params))
             for r in range(case["world"])]
    for s in slabs:
        s.set_flags(b.flags)
        if case["walls"]:
            s.set_walls(case["walls"])
        s.init_macro(f32(b.u0), rho=f32(b.rho0), c=f32(b.c0))
    sharding.step_local(slabs, steps)
    errs = {}
    for name in ("f", "u", "c"):
        got = np.concatenate([s.owned(getattr(s.dom.st, name).numpy()) for s in slabs],
                             axis=-3)
        errs[name] = float(np.abs(got - getattr(full.st, name).numpy()).max())
    return errs


@pytest.mark.parametrize("case", [
    dict(periodic=(True, True, True), world=3, walls=None, grad="lagged"),
    dict(periodic=(False, True, True), world=2, walls=None, grad="lagged"),
    dict(periodic=(False, False, False), world=3, walls=(False, False, True, True, True, True),
         grad="lagged"),
    dict(periodic=(True, False, False), world=4, walls=None, grad="local"),
])
def test_slab_cut_reproduces_the_undivided_oracle(case):
    errs = _run(case)
    assert max(errs.values()) <= 1e-14, errs


def test_slab_cut_with_the_directions_swapped_does_not():
    """Negative control: each halo filled with the 9 populations that point out of the
    receiving slab instead of into it."""
    old = dict(sharding.DIRECTION)
    try:
        sharding.DIRECTION.update({sharding.DOWN: +1, sharding.UP: -1})
        errs = _run(dict(periodic=(True, True, True), world=3, walls=None, grad="lagged"))
    finally:
        sharding.DIRECTION.update(old)
    assert errs["f"] > 1e-4, errs
