"""Pins of the far-field coupling (scales coarser than s0, Sec. 4.2.4 and 4.2.5) against
values fixed independently of the oracle's step code: the relaxation of a homogeneous
shear-stress state (the pull leaves a homogeneous state alone, the collision relaxes the
off-diagonal second moment by exactly 1 - S, and the far block's step is interpolated back
to t_n + dt_0 linearly), uniform flows, and the bookkeeping of scale boundaries."""
import numpy as np
import pytest
import torch

import synth
from oracle import cmr, coupling, grid


def _shear_state(shape, pi_xy):
    """Rest equilibrium plus the first-order non-equilibrium part of a pure xy stress,
    eps f^(1)_i = 9 w_i c_ix c_iy Pi_xy (zero mass and momentum), on every node."""
    Z, Y, X = shape
    feq = cmr.equilibrium(torch.ones(1, dtype=torch.float64), torch.zeros(1, 3, dtype=torch.float64))[0]
    w = feq.clone()                                   # rest equilibrium = lattice weights
    cx, cy = cmr.C[:, 0], cmr.C[:, 1]
    f1 = 9.0 * w * cx * cy * pi_xy
    return (feq + f1)[:, None, None, None].expand(27, Z, Y, X).clone()


def _pi_xy(f):
    return torch.einsum("q...,q->...", f, cmr.C[:, 0] * cmr.C[:, 1])


def test_far_block_relaxes_a_homogeneous_stress_by_one_minus_s_over_h():
    n0, h, nu0, pi0 = 10, 2.0, 0.02, 1e-3
    sc = synth.random_scene(dims=(n0, n0, n0), seed=1, periodic=(False, False, False), nu=nu0,
                            adaptive=False)
    b = sc.blocks[0]
    b.flags[:] = 0
    ms = coupling.MultiScale.build(sc)
    ms.blocks[0].state.f = _shear_state((n0, n0, n0), pi0)
    ms.blocks[0].state.u.zero_()
    nf = 12                                           # far block spans [-6, 16] at h = 2
    zeros = np.zeros((nf, nf, nf))
    i = ms.add_far_block((-6.0, -6.0, -6.0), h, (nf, nf, nf), np.ones_like(zeros),
                         np.zeros((3, nf, nf, nf)), zeros, np.zeros((nf, nf, nf), np.uint8))
    ms.blocks[i].state.f = _shear_state((nf, nf, nf), pi0)
    ms.step()
    s0 = 1.0 / (3.0 * nu0 + 0.5)
    sf = 1.0 / (3.0 * (nu0 / h) + 0.5)
    # s0 interior (two nodes or more from its scale boundary): one collision
    p0 = _pi_xy(ms.blocks[0].state.f)[2:-2, 2:-2, 2:-2]
    assert torch.allclose(p0, torch.full_like(p0, (1.0 - s0) * pi0), rtol=1e-12, atol=0)
    # far nodes away from s0: one own step, interpolated back with weight 1/h
    pf = _pi_xy(ms.blocks[i].state.f)
    away = torch.ones(nf, nf, nf, dtype=torch.bool)
    away[2:10, 2:10, 2:10] = False                    # nodes at -2 .. 12 touch s0's span
    assert torch.allclose(pf[away], torch.full_like(pf[away], (1.0 - sf / h) * pi0), rtol=1e-12,
                          atol=0)


def test_uniform_flow_stays_uniform_with_nested_far_blocks_and_a_refined_block():
    n0 = 12
    sc = synth.random_scene(dims=(n0, n0, n0), seed=2, periodic=(False, False, False), nu=0.01)
    b = sc.blocks[0]
    b.flags[:] = 0
    b.u0[:] = 0.0
    b.u0[0], b.u0[1] = 0.03, -0.02
    b.rho0[:] = 1.0
    ms = coupling.MultiScale.build(sc)
    u = np.zeros((3, 14, 14, 14))
    u[0], u[1] = 0.03, -0.02
    ones = np.ones((14, 14, 14))
    i1 = ms.add_far_block((-4.5, -4.5, -4.5), 1.5, (14, 14, 14), ones, u, 0 * ones,
                          np.zeros((14, 14, 14), np.uint8))
    u2 = np.zeros((3, 10, 10, 10))
    u2[0], u2[1] = 0.03, -0.02
    ones2 = np.ones((10, 10, 10))
    i2 = ms.add_far_block((-12.0, -12.0, -12.0), 4.0, (10, 10, 10), ones2, u2, 0 * ones2,
                          np.zeros((10, 10, 10), np.uint8))
    from oracle import dynamic
    dynamic.add_block_from_parent(ms, (2.0, 3.0, 2.5), 0.5, (10, 9, 11))
    assert ms.blocks[i1].child == 0 and ms.blocks[i2].child == i1
    for _ in range(3):
        ms.step()
    for blk in ms.blocks:
        uu = blk.state.u.reshape(3, -1)
        assert torch.allclose(uu[0], torch.full_like(uu[0], 0.03), atol=1e-13)
        assert torch.allclose(uu[1], torch.full_like(uu[1], -0.02), atol=1e-13)


def test_scale_boundary_bookkeeping():
    n0 = 8
    sc = synth.random_scene(dims=(n0, n0, n0), seed=3, periodic=(False, False, False),
                            inflow=(4, 4, 2.0, 0.05))
    ms = coupling.MultiScale.build(sc)
    fl0 = ms.blocks[0].state.flags.clone()
    z = np.zeros((8, 8, 8))
    with pytest.raises(ValueError):                   # does not contain s0
        ms.add_far_block((-1.0, -1.0, 0.5), 2.0, (8, 8, 8), z + 1, np.zeros((3, 8, 8, 8)), z,
                         np.zeros((8, 8, 8), np.uint8))
    ms.add_far_block((-2.0, -2.0, -2.0), 2.0, (8, 8, 8), z + 1, np.zeros((3, 8, 8, 8)), z,
                     np.zeros((8, 8, 8), np.uint8))
    fl = ms.blocks[0].state.flags
    outer = coupling.MultiScale._outer_layer((n0, n0, n0))
    inflow = (fl0 & grid.INFLOW) != 0
    ghost = (fl & grid.GHOST) != 0
    assert torch.equal(ghost, outer & ~inflow)        # inflow nodes keep their own update
    assert inflow[outer].any()
