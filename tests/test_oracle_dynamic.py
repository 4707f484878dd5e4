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


def test_visibility_of_a_cube_from_a_point_light():
    """One light point at (0, 24, 24) and an obstacle cube of voxels 20..27 on every axis
    (faces at 19.5 and 27.5): the segment from a node at x, off the light's axis by dy, dz,
    is off the axis by (dy, dz) x' / x where it crosses the plane x'.  It runs inside the
    cube's cross-section [-4.5, 3.5]^2 for all x' in [19.5, 27.5] when
    max(|dy|, |dz|) 27.5 / x < 3.5 (dark), and outside it for all x' when
    max(|dy|, |dz|) 19.5 / x > 4.5 (lit); one voxel of margin on each side for the voxel
    rounding.  Nodes upstream of the cube are all lit."""
    flags = np.zeros((48, 48, 64), np.uint8)
    flags[20:28, 20:28, 20:28] = grid.SOLID
    light = np.array([[0, 24, 24]])
    rng = np.random.default_rng(3)
    pts = np.stack([rng.integers(30, 64, 2000), rng.integers(0, 48, 2000),
                    rng.integers(0, 48, 2000)], 1)
    c = dynamic.visibility(flags, pts, light)
    x = pts[:, 0].astype(float)
    r = np.maximum(np.abs(pts[:, 1] - 24.0), np.abs(pts[:, 2] - 24.0))
    dark = r * 27.5 / x < 2.5
    lit = r * 19.5 / x > 5.5
    assert dark.sum() > 20 and lit.sum() > 20
    assert (c[dark] == 0).all() and (c[lit] == 1).all()
    up = np.stack([rng.integers(1, 19, 50), rng.integers(0, 48, 50), rng.integers(0, 48, 50)], 1)
    assert (dynamic.visibility(flags, up, light) == 1).all()


def test_light_samples_follow_the_inlet():
    flags = np.zeros((10, 12, 16), np.uint8)
    assert len(dynamic.light_samples(flags, 0, 16)) == 15       # 120 face nodes, every 8th
    flags[3:6, 4:8, 0] = grid.INFLOW
    ls = dynamic.light_samples(flags, 0, 4)
    assert len(ls) == 4 and (ls[:, 0] == 0).all()               # 12 inflow nodes, every 3rd
    assert set(map(tuple, ls[:, 1:])) <= {(y, z) for z in range(3, 6) for y in range(4, 8)}


def test_shadow_scales_worked_example():
    """Two light points, one each side of an obstacle plate: behind the plate the nodes that
    see neither light (c = 0) form the umbra of the finest scale, those that see one of the
    two the penumbra the coarser scale adds; with 3 scales (thresholds c <= 1 and c = 0)
    scale 2's wake box is the umbra's box and scale 1's the union with the penumbra's, and
    both include the obstacle box widened by d."""
    flags = np.zeros((9, 40, 48), np.uint8)
    flags[:, 16:24, 12:14] = grid.SOLID                        # plate x 12..13, y 16..23
    flags[4, 10, 0] = flags[4, 29, 0] = grid.INFLOW            # lights at y = 10 and y = 29
    lights = dynamic.light_samples(flags, 0, 16)
    assert len(lights) == 2
    sc = dynamic.shadow_scales(flags, 3, 0.5, 0.0, 20.0, flow_axis=0)
    zz, yy, xx = np.meshgrid(np.arange(9), np.arange(40), np.arange(48), indexing="ij")
    cand = (xx >= 12) & (xx <= 33) & ((flags & grid.SOLID) == 0)
    nodes = np.stack([xx[cand], yy[cand], zz[cand]], 1)
    c = dynamic.visibility(flags, nodes, lights)
    umbra, pen = nodes[c == 0], nodes[c <= 1]
    assert len(umbra) > 0 and len(pen) > len(umbra)
    (o1, h1, d1), (o2, h2, d2) = sc
    for (o, h, d), sel in (((o1, h1, d1), pen), ((o2, h2, d2), umbra)):
        for a in range(3):
            lo = min(float(sel[:, a].min()), [12, 16, 0][a])
            assert o[a] == max(lo, 0.0)
            hi = max(float(sel[:, a].max()), [13, 23, 8][a])
            top = [47, 39, 8][a]
            assert d[a] == max(int(math.floor((min(hi, top) - o[a]) / h + 1e-9)) + 1, 4)
