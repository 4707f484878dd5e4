"""The seeded input recipes the parity tests and the bench use, checked against their stated
shapes, sizes and value ranges (CPU)."""
import math

import numpy as np

import synth


def test_plume_recipe_scales_with_the_box():
    n = 128
    sc = synth.plume(n)
    b = sc.blocks[0]
    s = n / 256.0
    assert b.dims == (n, n, n) and sc.periodic == (False, False, False) and sc.nu == 1e-5
    solid = (b.flags & synth.SOLID) != 0
    z, y, x = np.nonzero(solid)
    r = 24 * s                                    # sphere of radius 24 at (72, n/2, n/2)
    assert np.allclose([x.mean(), y.mean(), z.mean()], [72 * s, n / 2, n / 2], atol=0.5)
    assert abs(solid.sum() / (4 / 3 * math.pi * r ** 3) - 1) < 0.05
    inflow = (b.flags & synth.INFLOW) != 0
    assert inflow[:, :, 1:].sum() == 0            # only on the x = 0 face
    assert abs(inflow.sum() / (math.pi * (16 * s) ** 2) - 1) < 0.05
    src = (b.flags & synth.SCALAR_SRC) != 0
    assert np.array_equal(src, inflow)             # the scalar source is the inflow disk
    ux = b.u0[0][inflow]
    assert np.all(np.abs(ux / 0.1 - 1) <= 0.01 + 1e-12) and ux.std() > 0   # +/- 1 % noise
    assert np.all(np.abs(b.u0[1:][:, inflow]) <= 0.001 + 1e-12)
    assert not b.u0[:, ~inflow].any()


def test_batch_recipe():
    scenes = synth.batch(64, seed=4)
    assert len(scenes) == 64
    L = np.array([s.blocks[0].dims[0] for s in scenes])
    assert L.min() >= 24 and L.max() <= 96
    assert all(s.blocks[0].dims == (l, l, l) for s, l in zip(scenes, L))
    # about 64 E[L^3] cells for L ~ U{24..96}
    assert abs((L ** 3).sum() / (64 * np.mean(np.arange(24, 97) ** 3)) - 1) < 0.15
    for s, l in zip(scenes, L):
        b = s.blocks[0]
        inflow = (b.flags & synth.INFLOW) != 0
        u = b.u0[0][inflow]
        assert 0.03 * 0.99 - 1e-12 <= u.min() and u.max() <= 0.1 * 1.01 + 1e-12
        solid = (b.flags & synth.SOLID) != 0
        assert solid.any()
        assert solid.sum() <= 4 * 4 / 3 * math.pi * (max(2.0, l / 8) + 1) ** 3


def test_multiscale_recipe_blocks_and_spheres():
    sc = synth.multiscale()
    dims = [b.dims for b in sc.blocks]
    assert dims == [(128,) * 3, (96,) * 3, (64,) * 3]
    assert [b.origin for b in sc.blocks] == [(0.0,) * 3, (24.0, 32.0, 32.0), (36.0, 50.0, 50.0)]
    assert np.allclose([b.h for b in sc.blocks], [1.0, 1 / 1.5, 1 / 2.25])
    s1 = sc.blocks[1]
    lo, hi = np.array(s1.origin), np.array(s1.origin) + (np.array(s1.dims) - 1) * s1.h
    z, y, x = np.nonzero(sc.blocks[0].flags & synth.SOLID)
    assert z.size > 0                              # the spheres lie inside s1's span
    pts = np.stack([x, y, z], 1)
    assert np.all(pts >= np.floor(lo)) and np.all(pts <= np.ceil(hi))
    inflow = (sc.blocks[0].flags & synth.INFLOW) != 0
    assert abs(sc.blocks[0].u0[0][inflow].mean() / 0.08 - 1) < 0.01


def test_taylor_green_and_adjoint_scene_recipes():
    tg = synth.taylor_green(32)
    assert tg.nu == 0.05 * 32 / 100 and abs(np.abs(tg.blocks[0].u0).max() - 0.05) < 1e-12
    sc, target = synth.adjoint_scene(n=32)
    b = sc.blocks[0]
    assert sc.periodic == (True, True, True)
    assert np.abs(b.u0).max() <= 0.05 + 1e-12
    peak = np.unravel_index(np.argmax(b.c0), b.c0.shape)
    assert peak == (16, 16, 16) and abs(b.c0.max() - 1) < 1e-12
    tpeak = np.array(np.unravel_index(np.argmax(target), target.shape))
    assert np.linalg.norm(tpeak - 16) <= 32 / 16 + math.sqrt(3) / 2 + 1e-9
