"""GPU parity of the no-slip wall faces (Sec. 6.1 second-order wall, regularized on-node
reading) against the FP64 oracle through the C-ABI: walls on faces, edges and corners,
with obstacles and an inflow disk in the block."""
import dataclasses

import numpy as np
import pytest

import synth
from oracle import grid
from tests.helpers import gpu_domain, gpu_state, max_err, oracle_params, oracle_state

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("walls", [(False, False, False, False, True, True),    # floor + lid
                                   (False, True, True, False, True, False),     # edges, corner
                                   (False, True, True, True, True, True)])      # five walls
def test_wall_faces_match_oracle(lib, walls):
    sc = synth.random_scene(dims=(26, 22, 18), seed=51, periodic=(False, False, False),
                            spheres=[(13.0, 11.0, 9.0, 3.0)], inflow=(11, 9, 3.0, 0.07), nu=0.01)
    b = sc.blocks[0]
    dom = gpu_domain(sc)
    dom.set_walls(walls)
    st = oracle_state(sc)
    p = dataclasses.replace(oracle_params(sc), walls=walls)
    for _ in range(8):
        dom.step(1)
        st = grid.step(st, p)
    f, u, c = gpu_state(dom, b.shape_zyx)
    umax = float(np.abs(st.u.numpy()).max())
    eu, ef, ec = max_err(u, st.u.numpy()), max_err(f, st.f.numpy()), max_err(c, st.c.numpy())
    print(f"walls {walls}: |du|={eu:.2e} (max|u| {umax:.3f}) |df|={ef:.2e} |dc|={ec:.2e}")
    assert eu <= 1e-5 * umax and ef <= 2e-7 and ec <= 1e-6
    # wall nodes (not inflow, not obstacle) are at rest
    z = np.zeros(b.shape_zyx, bool)
    if walls[4]:
        z[0] = True
    if walls[5]:
        z[-1] = True
    keep = z & ((b.flags & 3) == 0)
    assert np.abs(u[:, keep]).max() < 1e-7
    dom.close()


def test_wall_argument_checks(lib):
    from paper_1807_02284_gb300 import lbm
    dom = lbm.Domain((12, 12, 12), 0.01, periodic=(True, False, False))
    with pytest.raises(lbm.LBMError) as ei:
        dom.set_walls((True, False, False, False, False, False))   # x is periodic
    assert ei.value.status == lbm.LBM_ERR_INVALID_ARG
    dom.set_walls((False, False, False, False, True, True))
    dom.set_tape(2)                                  # the adjoint covers wall faces
    dom.set_tape(0)
    dom.set_walls((False,) * 6)
    dom.step(2)
    dom.sync()
    dom.close()


@pytest.mark.parametrize("faces", [(False,) * 6, (False, False, False, False, True, False)])
def test_obstacle_surface_walls_match_oracle(lib, faces):
    """Obstacle surfaces as regularized on-node walls (Sec. 6.1 wall on objects): two spheres
    (one touching the floor when the floor is a wall; the r = 3 one has surface voxels with
    no inner neighbour), a plate one voxel thick, an inflow disk, open faces, low viscosity."""
    from paper_1807_02284_gb300 import lbm
    sc = synth.random_scene(dims=(28, 22, 18), seed=53, periodic=(False, False, False),
                            spheres=[(14.0, 11.0, 9.0, 3.0), (21.0, 7.0, 2.0, 2.5)],
                            inflow=(11, 9, 3.0, 0.07), nu=1e-4)
    b = sc.blocks[0]
    b.flags[6:12, 12:18, 23] |= synth.SOLID          # the plate (no inner voxels at all)
    b.rho0[b.flags & synth.SOLID != 0] = 1.0
    dom = gpu_domain(sc)
    dom.set_walls(faces, obstacles=True)
    dom.init_macro(np.asarray(b.u0, np.float32), rho=np.asarray(b.rho0, np.float32),
                   c=np.asarray(b.c0, np.float32))
    st = oracle_state(sc)
    p = dataclasses.replace(oracle_params(sc), walls=faces, obstacle_walls=True)
    surf = grid.surface_voxels(st.flags, sc.periodic).numpy()
    fl = dom.read_field(lbm.LBM_FIELD_FLAGS, lbm.LBM_U8).reshape(b.shape_zyx)
    assert np.array_equal((fl & 64) != 0, surf)
    assert np.array_equal((fl & 1) != 0, ((b.flags & 1) != 0) & ~surf)
    for _ in range(8):
        dom.step(1)
        st = grid.step(st, p)
    f, u, c = gpu_state(dom, b.shape_zyx)
    umax = float(np.abs(st.u.numpy()).max())
    eu, ef, ec = max_err(u, st.u.numpy()), max_err(f, st.f.numpy()), max_err(c, st.c.numpy())
    print(f"obstacle walls {faces}: |du|={eu:.2e} (max|u| {umax:.3f}) |df|={ef:.2e} |dc|={ec:.2e}")
    assert eu <= 1e-5 * umax and ef <= 2e-7 and ec <= 1e-6
    assert np.abs(u[:, surf]).max() < 1e-6          # the wall nodes are at rest
    dom.close()


def test_obstacle_walls_follow_new_flags_and_can_be_switched_off(lib):
    """Flags set after the wall mode get their surfaces derived; switching the mode off
    restores every obstacle voxel to halfway bounce-back (bit 0)."""
    import torch
    from paper_1807_02284_gb300 import lbm
    sc = synth.random_scene(dims=(16, 16, 16), seed=54, periodic=(True, True, True),
                            spheres=[(8.0, 8.0, 8.0, 3.5)])
    b = sc.blocks[0]
    dom = lbm.Domain(b.dims, sc.nu, periodic=sc.periodic)
    dom.set_walls((False,) * 6, obstacles=True)
    dom.set_flags(b.flags)
    surf = grid.surface_voxels(torch.as_tensor(b.flags), sc.periodic).numpy()
    fl = dom.read_field(lbm.LBM_FIELD_FLAGS, lbm.LBM_U8).reshape(b.shape_zyx)
    assert surf.any() and np.array_equal((fl & 64) != 0, surf)
    dom.set_walls((False,) * 6)
    fl = dom.read_field(lbm.LBM_FIELD_FLAGS, lbm.LBM_U8).reshape(b.shape_zyx)
    assert not (fl & 64).any() and np.array_equal((fl & 1) != 0, (b.flags & 1) != 0)
    dom.close()


def test_obstacle_wall_argument_checks(lib):
    from paper_1807_02284_gb300 import lbm
    dom = lbm.Domain((16, 16, 16), 0.01, periodic=(False, False, False))
    dom.set_walls((False,) * 6, obstacles=True)
    dom.set_tape(2)                                  # the adjoint covers obstacle walls
    dom.set_tape(0)
    dom.add_scale_block((4.0, 4.0, 4.0), 0.5, (8, 8, 8))   # refined blocks take them too
    with pytest.raises(lbm.LBMError) as ei:          # but not their adjoint
        dom.set_tape(2)
    assert ei.value.status == lbm.LBM_ERR_UNSUPPORTED
    with pytest.raises(lbm.LBMError) as ei:          # nor blocks started from their parent
        dom.init_block_from_parent(1)
    assert ei.value.status == lbm.LBM_ERR_UNSUPPORTED
    dom.set_walls((False,) * 6)
    dom.set_walls((False,) * 6, obstacles=True)
    dom.step(2)
    dom.sync()
    dom.close()


def test_regularized_sphere_stays_bounded_at_high_reynolds_number(lib):
    """The flow past a sphere at nu = 1e-4 (196 x 98 x 98, inflow 0.1): with the sphere's
    surface as regularized walls the run stays finite and bounded for 2000 steps (with
    halfway bounce-back on the same sphere it blows up within 1000 steps)."""
    import torch
    from paper_1807_02284_gb300 import lbm
    sc = synth.ringing_channel()
    b = sc.blocks[0]
    dom = gpu_domain(sc)
    dom.set_walls((False,) * 6, obstacles=True)
    dom.init_macro(np.asarray(b.u0, np.float32), rho=np.asarray(b.rho0, np.float32),
                   c=np.asarray(b.c0, np.float32))
    u = torch.empty(3 * b.flags.size, dtype=torch.float32, device="cuda")
    for _ in range(8):
        dom.step(250)
        dom.read_field(lbm.LBM_FIELD_U, lbm.LBM_F32, out=u)   # raises LBM_ERR_DIVERGED on a blow-up
        dom.sync()
        assert float(u.abs().max()) < 0.75
    dom.close()
