"""Exact pin of the oracle's Algorithm 1 time bookkeeping (Sec. 4.2.4, Sec. 4.2.5, Algorithm 1).

A uniform equilibrium flow U carries a passive scalar that is affine in space,
c(x, 0) = c0 + G . x (x in reference units).  The exact solution is c(x, t) = c0 + G . (x - U t)
with t in reference steps: velocity is the same number on every scale (dt_s = dx_s), so a
sub-step of a block of spacing h moves the scalar by U h reference units in h reference time.
Every operation of the coupled schedule is exact on these data:
  * the semi-Lagrangian step samples trilinearly, which reproduces affine fields;
  * prior-mapping (trilinear in space, linear in time between t_n and t_n + dt_0) sees a
    field that is affine in space and linear in time at every fixed point;
  * the three-point Lagrange alignment through t_n, t_n + (l-1) h and t_n + l h is exact on
    anything linear in time;
  * post-mapping and the far-field lerp (1 - 1/h, 1/h) are exact for the same reasons;
  * the populations stay the uniform equilibrium (a fixed point of every step and mapping).
So after reference step n every interior and scale-boundary node of every block must hold
c0 + G . (x - U n) to rounding, except where an upstream open face of the outermost block
(whose departure point is clamped into the block) has had time to reach: one node per step.

A schedule slip breaks the identity: a ghost layer mapped at t_n + j h instead of
t_n + (j - 1) h, an alignment fed the wrong pair of levels, or a far block left at its own
t_n + h dt_0 instead of being interpolated back to t_n + dt_0.  The negative controls below
plant each slip in the oracle and check that the pin catches it.

U and G are exact binary fractions, so the float32-rounded inputs that far blocks receive are
the same numbers."""
import numpy as np
import pytest
import torch

import synth
from oracle import coupling, grid

U = np.array([0.0625, -0.046875, 0.03125])
G = np.array([0.0625, -0.046875, 0.03125])
C0 = 0.25
TOL = 1e-12


def affine_block(dims, origin=(0.0, 0.0, 0.0), h=1.0):
    b = synth._empty_block(dims, origin=origin, h=h)
    xs, ys, zs = b.node_coords()
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    for a in range(3):
        b.u0[a] = U[a]
    b.c0[:] = C0 + G[0] * X + G[1] * Y + G[2] * Z
    return b


def exact_scalar(origin, h, dims, t):
    nx, ny, nz = dims
    xs = origin[0] + h * np.arange(nx) - U[0] * t
    ys = origin[1] + h * np.arange(ny) - U[1] * t
    zs = origin[2] + h * np.arange(nz) - U[2] * t
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    return C0 + G[0] * X + G[1] * Y + G[2] * Z


def upstream_margin(dims, n):
    """Nodes of an open-faced block that no upstream face has reached after n steps (the
    contamination moves one node per step against the flow on each axis)."""
    nx, ny, nz = dims
    keep = np.ones((nz, ny, nx), bool)
    for a, size in enumerate((nx, ny, nz)):
        sl = [slice(None)] * 3
        ax = 2 - a
        if U[a] > 0:
            sl[ax] = slice(0, min(n, size))
        elif U[a] < 0:
            sl[ax] = slice(max(size - n, 0), size)
        keep[tuple(sl)] = False
    return keep


def nested_scene():
    """s0 22^3 (open faces), s1 at h = 1/1.5 and s2 at h = 1/2.25 nested inside s1."""
    s0 = affine_block((22, 22, 22))
    s1 = affine_block((14, 13, 12), origin=(6.0, 5.5, 6.25), h=1 / 1.5)
    s2 = affine_block((9, 9, 9), origin=(8.0, 7.5, 8.0), h=1 / 2.25)
    return synth.Scene(blocks=[s0, s1, s2], periodic=(False, False, False), nu=0.01)


def far_scene():
    """s0 16^3 inside a far block at h = 2 (10 reference units of padding), with a refined
    block at h = 1/1.5 inside s0."""
    s0 = affine_block((16, 16, 16))
    s1 = affine_block((11, 10, 10), origin=(4.0, 4.5, 3.5), h=1 / 1.5)
    far = affine_block((19, 19, 19), origin=(-10.0, -10.0, -10.0), h=2.0)
    return synth.Scene(blocks=[s0, s1], periodic=(False, False, False), nu=0.01), far


def build(kind):
    if kind == "nested":
        return coupling.MultiScale.build(nested_scene(), f32_inputs=False)
    sc, far = far_scene()
    ms = coupling.MultiScale.build(sc, f32_inputs=False)
    ms.add_far_block(far.origin, far.h, far.dims, far.rho0, far.u0, far.c0, far.flags)
    return ms


def checked_masks(ms, n):
    """Per block, the nodes held to the closed form after n reference steps."""
    masks = []
    has_far = any(b.far for b in ms.blocks)
    for b in ms.blocks:
        shape = tuple(reversed(b.dims))
        if b.far or (b.h == 1.0 and not has_far):
            masks.append(upstream_margin(b.dims, n))       # the outermost block's open faces
        else:
            masks.append(np.ones(shape, bool))
    return masks


def schedule_errors(ms, steps):
    """Largest deviation from the closed form per reference step (every checked node of every
    block, interior and scale boundary alike)."""
    errs = []
    for n in range(1, steps + 1):
        ms.step()
        worst = 0.0
        for b, m in zip(ms.blocks, checked_masks(ms, n)):
            want = exact_scalar(b.origin, b.h, b.dims, n)
            got = b.state.c.numpy()
            worst = max(worst, float(np.abs(got - want)[m].max()))
        errs.append(worst)
    return errs


def test_affine_scalar_case_fits_the_tolerance_argument():
    """The scene is what the pin assumes: every block's velocity is U, every mapping is
    exercised (ghost layers, post-mapped nodes, and for the far case an overlap and an outer
    layer), and the non-integer ratios need sub-steps with temporal interpolation."""
    ms = build("nested")
    assert [b.substeps for b in ms.blocks] == [1, 2, 3]
    assert [b.integer_ratio for b in ms.blocks] == [True, False, False]
    assert [b.parent for b in ms.blocks[1:]] == [0, 1]
    msf = build("far")
    assert [b.far for b in msf.blocks] == [False, False, True]
    assert bool(((msf.blocks[0].state.flags & coupling.GHOST) != 0).any())
    for b in ms.blocks + msf.blocks:
        assert np.allclose(b.state.u.numpy().reshape(3, -1), U[:, None], atol=0)


@pytest.mark.parametrize("kind", ["nested", "far"])
def test_algorithm1_schedule_is_exact_on_affine_scalar_transport(kind):
    errs = schedule_errors(build(kind), 3)
    assert max(errs) < TOL, errs
    # and the flow itself stays the uniform equilibrium
    ms = build(kind)
    ms.run(2)
    for b in ms.blocks:
        rho, u = grid.macros_field(b.state)
        assert float((u - torch.as_tensor(U)[:, None, None, None]).abs().max()) < 1e-14
        assert float((rho - 1.0).abs().max()) < 1e-14


def test_negative_control_ghost_layer_one_substep_late(monkeypatch):
    """Prior-mapping at theta = j h (the end of sub-step j) instead of (j - 1) h."""
    orig = coupling.MultiScale.prior_map

    def late(self, i, theta, saved):
        if theta < 1.0:
            theta = theta + self.blocks[i].h
        return orig(self, i, theta, saved)

    monkeypatch.setattr(coupling.MultiScale, "prior_map", late)
    errs = schedule_errors(build("nested"), 2)
    assert max(errs) > 1e3 * TOL, errs


def test_negative_control_alignment_from_swapped_levels(monkeypatch):
    """Alignment fed the t_n + l h level where it expects t_n + (l - 1) h, and vice versa."""
    orig = coupling.MultiScale.align

    def swapped(self, b, s0, s_prev, s_last):
        return orig(self, b, s0, s_last, s_prev)

    monkeypatch.setattr(coupling.MultiScale, "align", swapped)
    errs = schedule_errors(build("nested"), 2)
    assert max(errs) > 1e3 * TOL, errs


def test_negative_control_alignment_from_the_unrefreshed_start(monkeypatch):
    """Alignment fed the start level twice (t_n in place of t_n + (l - 1) h)."""
    orig = coupling.MultiScale.align

    def stale(self, b, s0, s_prev, s_last):
        return orig(self, b, s0, s0, s_last)

    monkeypatch.setattr(coupling.MultiScale, "align", stale)
    errs = schedule_errors(build("nested"), 2)
    assert max(errs) > 1e3 * TOL, errs


def test_negative_control_far_block_not_interpolated_back(monkeypatch):
    """A far block left at its own t_n + h dt_0 instead of t_n + dt_0."""
    def unaligned(self, i):
        b = self.blocks[i]
        b.state = grid.step(b.state, b.params)

    monkeypatch.setattr(coupling.MultiScale, "far_step", unaligned)
    errs = schedule_errors(build("far"), 2)
    assert max(errs) > 1e3 * TOL, errs


def test_negative_control_scale_boundary_from_the_far_block_at_t_n(monkeypatch):
    """s0's scale boundary mapped from the far block's state at t_n (before its step) instead
    of its state at t_n + dt_0."""
    orig_out = coupling.MultiScale.far_out_map
    orig_far = coupling.MultiScale.far_step
    stash = {}

    def keep_old(self, i):
        stash[i] = self.blocks[i].state.clone()
        orig_far(self, i)

    def from_old(self, i):
        new = self.blocks[i].state
        self.blocks[i].state = stash[i]
        orig_out(self, i)
        self.blocks[i].state = new

    monkeypatch.setattr(coupling.MultiScale, "far_step", keep_old)
    monkeypatch.setattr(coupling.MultiScale, "far_out_map", from_old)
    errs = schedule_errors(build("far"), 2)
    assert max(errs) > 1e3 * TOL, errs
