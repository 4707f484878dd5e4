"""Pins of the dynamic-scale oracle (Sec. 5) against values fixed independently of its code:
closed forms of central differences of sinusoids, hand-computed placements, hand-derived
nearest-node obstacles, and the exactness of the mapping on equilibrium states."""
import math

import numpy as np
import pytest
import torch

import synth
from oracle import cmr, coupling, dynamic, grid


def _sin_shear_state(X, Y, Z, U0, A, solid=()):
    """u_x = U0 + A sin(ky y) sin(kz z) on a periodic box, u_y = u_z = 0."""
    ky, kz = 2 * math.pi / Y, 2 * math.pi / Z
    z, y, x = np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    u = np.zeros((3, Z, Y, X))
    u[0] = U0 + A * np.sin(ky * y) * np.sin(kz * z)
    flags = np.zeros((Z, Y, X), np.uint8)
    for (sx, sy, sz) in solid:     # velocity left analytic so neighbours keep the closed form
        flags[sz, sy, sx] = grid.SOLID
    st = grid.State(torch.zeros((27, Z, Y, X), dtype=torch.float64), torch.as_tensor(u),
                    torch.zeros((Z, Y, X), dtype=torch.float64), torch.as_tensor(flags))
    return st, ky, kz, (z, y, x)


def test_detection_matches_the_closed_form_of_central_differences():
    X, Y, Z, U0, A = 10, 24, 18, 0.02, 0.05
    st, ky, kz, (z, y, x) = _sin_shear_state(X, Y, Z, U0, A, solid=[(3, 6, 2)])
    # half central differences of sin are exact: (sin(k(n+1)) - sin(k(n-1))) / 2 = cos(kn) sin(k)
    dy = A * math.sin(ky) * np.cos(ky * y) * np.sin(kz * z)
    dz = A * math.sin(kz) * np.sin(ky * y) * np.cos(kz * z)
    g_exact = np.sqrt(dy ** 2 + dz ** 2)
    u_exact = np.abs(U0 + A * np.sin(ky * y) * np.sin(kz * z))
    g_thr, u_thr = 0.55 * g_exact.max(), 0.045
    sel = (g_exact >= g_thr) & (u_exact >= u_thr)
    assert sel[2, 6, 3]
    sel[2, 6, 3] = False                                  # the obstacle voxel is never kept
    # no sample sits on a threshold, so the decision is the same in any precision
    assert np.abs(g_exact - g_thr).min() > 1e-6 and np.abs(u_exact - u_thr).min() > 1e-6
    n, box, g, umag = dynamic.detect(st, (True, True, True), g_thr, u_thr)
    zz, yy, xx = np.nonzero(sel)
    assert n == int(sel.sum()) > 0
    assert box == (int(xx.min()), int(yy.min()), int(zz.min()),
                   int(xx.max()), int(yy.max()), int(zz.max()))
    ok = np.ones_like(sel)
    ok[2, 6, 3] = False
    assert np.allclose(g.numpy()[ok], g_exact[ok], atol=1e-15)


def test_detection_thresholds_select_nothing_above_the_maximum():
    st, _, _, _ = _sin_shear_state(8, 16, 16, 0.0, 0.05)
    n, box, _, _ = dynamic.detect(st, (True, True, True), 1.0, 0.0)
    assert n == 0 and box is None


@pytest.mark.parametrize("case", [
    # box, src origin, src h, h, margin, ref dims -> origin, dims (worked by hand)
    ((10, 20, 30, 40, 50, 60), (0, 0, 0), 1.0, 0.5, 2, (128, 128, 128),
     (8.0, 18.0, 28.0), (69, 69, 69)),
    # clipped at the lower and upper ends: x [-3, 6] -> [0, 6]; z [117, 130] -> [117, 127]
    ((0, 0, 120, 3, 3, 127), (0, 0, 0), 1.0, 0.4, 3, (64, 64, 128),
     (0.0, 0.0, 117.0), (16, 16, 26)),
    # a single sample: at least 4 nodes; near the top the box is shifted down
    ((5, 7, 5, 5, 7, 5), (0, 0, 0), 1.0, 0.5, 0, (8, 8, 8),
     (5.0, 5.5, 5.0), (4, 4, 4)),
    # detection on a refined block (origin 10, spacing 0.5)
    ((2, 4, 6, 10, 12, 14), (10, 10, 10), 0.5, 0.25, 1, (64, 64, 64),
     (10.5, 11.5, 12.5), (21, 21, 21)),
])
def test_placement_worked_examples(case):
    box, so, sh, h, m, ref, origin, dims = case
    o, d = dynamic.place(box, so, sh, h, m, ref)
    assert d == dims
    assert np.allclose(o, origin, atol=1e-12)


def test_nearest_node_obstacles_and_ghost_layer():
    """Coarse obstacle at node (5,5,5); fine nodes at 3.25 + 0.5 i whose nearest coarse node
    is 5 are i = 3 (4.75) and i = 4 (5.25)."""
    sc = synth.random_scene(dims=(12, 12, 12), seed=1, periodic=(False, False, False))
    ms = coupling.MultiScale.build(sc)
    ms.blocks[0].state.flags[:] = 0
    ms.blocks[0].state.flags[5, 5, 5] = grid.SOLID
    fl = dynamic.nearest_flags(ms.blocks[0], (3.25, 3.25, 3.25), 0.5, (10, 10, 10))
    solid = (fl & grid.SOLID) != 0
    expect = np.zeros((10, 10, 10), bool)
    expect[3:5, 3:5, 3:5] = True
    assert np.array_equal(solid, expect)
    ghost = (fl & grid.GHOST) != 0
    assert ghost[0].all() and ghost[-1].all() and ghost[:, 0].all() and ghost[:, :, -1].all()
    assert not ghost[1:-1, 1:-1, 1:-1].any()


def test_new_block_of_a_uniform_flow_is_its_exact_equilibrium_and_stays_uniform():
    """The mapping keeps rho and u and scales only the non-equilibrium part, so a block
    started from a uniform equilibrium flow is that equilibrium at every node; stepping the
    two-block domain keeps it uniform."""
    n = 16
    sc = synth.random_scene(dims=(n, n, n), seed=2, periodic=(True, True, True))
    b = sc.blocks[0]
    b.flags[:] = 0
    b.u0[:] = 0.0
    b.u0[0] = 0.04
    b.u0[2] = -0.01
    b.rho0[:] = 1.0
    ms = coupling.MultiScale.build(sc)
    i = dynamic.add_block_from_parent(ms, (3.0, 4.0, 2.5), 1 / 1.5, (10, 9, 11))
    nb = ms.blocks[i]
    assert nb.parent == 0 and nb.substeps == 2
    feq = cmr.equilibrium(torch.ones(1, dtype=torch.float64),
                          torch.tensor([[0.04, 0.0, -0.01]], dtype=torch.float64))[0]
    f = nb.state.f.reshape(27, -1)
    assert torch.allclose(f, feq[:, None].expand_as(f), atol=1e-14)
    for _ in range(3):
        ms.step()
    for blk in ms.blocks:
        u = blk.state.u.reshape(3, -1)
        assert torch.allclose(u[0], torch.full_like(u[0], 0.04), atol=1e-13)
        assert torch.allclose(u[2], torch.full_like(u[2], -0.01), atol=1e-13)
    dynamic.remove_last_block(ms)
    assert len(ms.blocks) == 1


def test_static_scales_worked_example():
    """Obstacle voxels spanning x 10..14, y 20..23, z 5..9 in a 64 x 48 x 32 block; 3 scales
    with h_min = 0.5, d_max = 8, wake 12 along x (worked by hand):
      scale 1: h = 0.75, d = 4: x [6, 30], y [16, 27], z [1, 13] -> 33, 15, 17 nodes;
      scale 2: h = 0.5,  d = 0: x [10, 26], y [20, 23], z [5, 9]  -> 33, 7, 9 nodes."""
    flags = np.zeros((32, 48, 64), np.uint8)
    flags[5:10, 20:24, 10:15] = grid.SOLID
    sc = dynamic.static_scales(flags, 3, 0.5, 8.0, 12.0, flow_axis=0)
    assert len(sc) == 2
    (o1, h1, d1), (o2, h2, d2) = sc
    assert h1 == 0.75 and d1 == (33, 15, 17) and np.allclose(o1, (6.0, 16.0, 1.0))
    assert h2 == 0.5 and d2 == (33, 7, 9) and np.allclose(o2, (10.0, 20.0, 5.0))
    assert dynamic.static_scales(np.zeros((8, 8, 8), np.uint8), 3, 0.5, 4.0, 0.0) == []
