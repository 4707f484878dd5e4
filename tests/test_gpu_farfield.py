"""GPU parity of the far-field coupling (scales coarser than s0, Sec. 4.2.4-4.2.5) against
the FP64 oracle through the C-ABI: a far block around the reference block, nested far
blocks with a refined block inside s0, the scale-boundary flags, and argument checks."""
import numpy as np
import pytest

import synth
from oracle import coupling, dynamic
from tests.helpers import f32
from tests.test_gpu_multiscale import compare, gpu_multiscale

pytestmark = pytest.mark.gpu


def _scene():
    return synth.random_scene(dims=(20, 18, 16), seed=41, periodic=(False, False, False),
                              spheres=[(11.0, 9.0, 8.0, 2.5)], inflow=(9, 8, 3.0, 0.08), nu=0.004)


def _add_far(dom, ms, inner, h, pad, seed):
    fb = synth.far_block(inner, h, pad, seed=seed, amp=0.03)
    fid = dom.add_scale_block(fb.origin, fb.h, fb.dims)
    dom.set_flags(fb.flags, block=fid)
    dom.init_macro(f32(fb.u0), rho=f32(fb.rho0), c=f32(fb.c0), block=fid)
    oid = ms.add_far_block(fb.origin, fb.h, fb.dims, fb.rho0, fb.u0, fb.c0, fb.flags)
    assert fid == oid
    return fid, fb


def test_far_block_around_the_reference_block(lib):
    from paper_1807_02284_gb300 import lbm
    sc = _scene()
    dom = gpu_multiscale(sc)
    ms = coupling.MultiScale.build(sc)
    fid, fb = _add_far(dom, ms, sc.blocks[0], 1.5, 6.0, seed=5)
    i = dom.info(fid)
    assert i.h == 1.5 and i.substeps == 1
    fl = dom.read_field(lbm.LBM_FIELD_FLAGS, lbm.LBM_U8, 0).reshape(sc.blocks[0].shape_zyx)
    assert np.array_equal(fl & 8, ms.blocks[0].state.flags.numpy() & 8)
    for n in range(4):
        dom.step(1)
        ms.step()
    compare(dom, ms, "far field")
    dom.close()


def test_nested_far_blocks_with_a_refined_block(lib):
    sc = _scene()
    dom = gpu_multiscale(sc)
    ms = coupling.MultiScale.build(sc)
    f1, fb1 = _add_far(dom, ms, sc.blocks[0], 1.5, 4.5, seed=6)
    f2, _ = _add_far(dom, ms, fb1, 3.0, 6.0, seed=7)
    origin, h, dims = (4.0, 3.5, 3.0), 0.5, (20, 18, 16)
    rid = dom.add_scale_block(origin, h, dims)
    dom.init_block_from_parent(rid)
    assert dynamic.add_block_from_parent(ms, origin, h, dims) == rid == 3
    for n in range(3):
        dom.step(1)
        ms.step()
    compare(dom, ms, "nested far field + refined")
    dom.step(5)                                   # graph-captured chunk with far blocks
    for n in range(5):
        ms.step()
    compare(dom, ms, "nested far field + refined, captured")
    dom.close()


def test_scale_boundary_flags_follow_far_blocks(lib):
    from paper_1807_02284_gb300 import lbm
    sc = _scene()
    b0 = sc.blocks[0]
    dom = gpu_multiscale(sc)
    outer = np.zeros(b0.shape_zyx, bool)
    outer[0], outer[-1], outer[:, 0], outer[:, -1], outer[:, :, 0], outer[:, :, -1] = (True,) * 6
    fb = synth.far_block(b0, 2.0, 4.0, seed=3)
    fid = dom.add_scale_block(fb.origin, fb.h, fb.dims)
    fl = dom.read_field(lbm.LBM_FIELD_FLAGS, lbm.LBM_U8, 0).reshape(b0.shape_zyx)
    keep = (b0.flags & (1 | 2)) != 0
    assert np.array_equal((fl & 8) != 0, outer & ~keep)
    dom.set_flags(b0.flags)                        # user flags again: the boundary stays
    fl = dom.read_field(lbm.LBM_FIELD_FLAGS, lbm.LBM_U8, 0).reshape(b0.shape_zyx)
    assert np.array_equal((fl & 8) != 0, outer & ~keep)
    dom.remove_scale_block(fid)                    # open faces again
    fl = dom.read_field(lbm.LBM_FIELD_FLAGS, lbm.LBM_U8, 0).reshape(b0.shape_zyx)
    assert not (fl & 8).any()
    dom.step(3)
    dom.sync()
    dom.close()


def test_far_block_argument_checks(lib):
    from paper_1807_02284_gb300 import lbm
    sc = _scene()
    dom = gpu_multiscale(sc)
    with pytest.raises(lbm.LBMError) as ei:        # does not contain the reference block
        dom.add_scale_block((-2.0, -2.0, 1.0), 2.0, (14, 14, 14))
    assert ei.value.status == lbm.LBM_ERR_INVALID_ARG
    with pytest.raises(lbm.LBMError) as ei:        # h = 1 is the reference scale
        dom.add_scale_block((0.0, 0.0, 0.0), 1.0, (20, 18, 16))
    assert ei.value.status == lbm.LBM_ERR_INVALID_ARG
    dom.close()
    per = lbm.Domain((12, 12, 12), 0.01, periodic=(True, True, True))
    with pytest.raises(lbm.LBMError) as ei:
        per.add_scale_block((-4.0, -4.0, -4.0), 2.0, (11, 11, 11))
    assert ei.value.status == lbm.LBM_ERR_UNSUPPORTED
    per.close()


@pytest.mark.parametrize("walls_first", [True, False])
def test_far_block_with_obstacle_walls(lib, walls_first):
    """The open-boundary setting of Sec. 4.2.4 / 6.1 with the second-order wall on the
    obstacle's surface: a far block around s0 whose sphere is a regularized wall (the far
    block keeps halfway bounce-back for its own obstacle voxels, which s0 overwrites); parity
    with the oracle for both orders of setting the walls and adding the far block.  Wall
    faces and far-field blocks still exclude each other."""
    from paper_1807_02284_gb300 import lbm
    from oracle import grid
    sc = _scene()
    dom = gpu_multiscale(sc)
    b0 = sc.blocks[0]

    def walls():
        dom.set_walls((False,) * 6, obstacles=True)
        dom.init_macro(f32(b0.u0), rho=f32(b0.rho0), c=f32(b0.c0), block=0)
    ms = coupling.MultiScale.build(sc, obstacle_walls=True)
    if walls_first:
        walls()
        fid, fb = _add_far(dom, ms, b0, 1.5, 6.0, seed=5)
    else:
        fid, fb = _add_far(dom, ms, b0, 1.5, 6.0, seed=5)
        walls()
    s = grid.surface_voxels(ms.blocks[0].state.flags, ms.blocks[0].params.periodic)
    fl = dom.read_field(lbm.LBM_FIELD_FLAGS, lbm.LBM_U8, 0).reshape(b0.shape_zyx)
    assert s.sum() > 0 and np.array_equal((fl & 64) != 0, s.numpy())
    ffl = dom.read_field(lbm.LBM_FIELD_FLAGS, lbm.LBM_U8, fid).reshape(fb.shape_zyx)
    assert not (ffl & 64).any()                      # the far block has no wall nodes
    assert np.array_equal(fl & 8, ms.blocks[0].state.flags.numpy() & 8)
    for _ in range(4):
        dom.step(1)
        ms.step()
    compare(dom, ms, f"far field + obstacle walls (walls first {walls_first})")
    with pytest.raises(lbm.LBMError) as ei:
        dom.set_walls((False, False, False, False, True, False), obstacles=True)
    assert ei.value.status == lbm.LBM_ERR_UNSUPPORTED
    dom.close()
