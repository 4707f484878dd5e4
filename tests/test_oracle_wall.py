"""Pins of the second-order no-slip wall on flat block faces (Sec. 6.1; read as the
regularized on-node wall of the cited method): second-order convergence of the decay of a
shear mode between two walls to the Navier-Stokes rate, the exact parabolic curvature of a
body-forced channel, and the wall-node invariants (mass from the known populations, zero
momentum, the non-equilibrium stress of the completed set kept).  The same wall on the
surface voxels of obstacles: hand-counted surface voxels, the channel between obstacle
slabs (the exact curvature, and the same state as the channel between wall faces), and the
invariants on a voxel with unknown populations from several directions."""
import math

import numpy as np
import torch

from oracle import cmr, grid

WALLS_Z = (False,) * 4 + (True, True)


def _shear_decay_rate_error(H, nu=0.05, U=1e-3):
    Z = H + 1
    z = np.arange(Z)
    u0 = np.zeros((3, Z, 1, 1))
    u0[0, :, 0, 0] = U * np.sin(math.pi * z / H)      # zero on the wall nodes z = 0, H
    st = grid.init_state(np.ones((Z, 1, 1)), u0, np.zeros((Z, 1, 1)), np.zeros((Z, 1, 1), np.uint8))
    p = grid.Params(nu=nu, periodic=(True, True, False), adaptive=False, walls=WALLS_Z)
    basis = np.sin(math.pi * z / H)
    t0, t1 = int(0.2 * H * H / nu), int(0.6 * H * H / nu)
    amps = {}
    for t in range(1, t1 + 1):
        st = grid.step(st, p)
        if t in (t0, t1):
            amps[t] = float((st.u[0, :, 0, 0].numpy() * basis).sum() / (basis * basis).sum())
    rate = -math.log(amps[t1] / amps[t0]) / (t1 - t0)
    return rate / (nu * math.pi ** 2 / H ** 2) - 1.0


def test_shear_mode_decay_converges_at_second_order_to_the_navier_stokes_rate():
    """u_x = U sin(pi z / H) between on-node walls at z = 0 and z = H decays at
    nu (pi / H)^2; the error of the lattice rate falls 4x per doubling of H."""
    e8, e16 = _shear_decay_rate_error(8), _shear_decay_rate_error(16)
    assert abs(e16) < 5e-3
    assert 3.6 < e8 / e16 < 4.4, (e8, e16)


def test_body_forced_channel_profile_has_the_exact_curvature():
    """Steady body-forced channel between the walls: away from the wall nodes the profile
    is a parabola of curvature -g / nu exactly (the forcing shifts it by a constant)."""
    H, nu, g = 8, 0.2, 1e-5
    Z = H + 1
    st = grid.init_state(np.ones((Z, 1, 1)), np.zeros((3, Z, 1, 1)), np.zeros((Z, 1, 1)),
                         np.zeros((Z, 1, 1), np.uint8))
    p = grid.Params(nu=nu, periodic=(True, True, False), adaptive=False, body_force=(g, 0.0, 0.0),
                    walls=WALLS_Z)
    for _ in range(int(8 * H * H / nu)):
        st = grid.step(st, p)
    u = st.u[0, :, 0, 0].numpy()
    d2 = u[3:-1] - 2 * u[2:-2] + u[1:-3]            # z = 2 .. H-2: neighbours are interior nodes
    assert np.allclose(d2, -g / nu, rtol=1e-6)
    assert u[0] == 0.0 and u[-1] == 0.0


def test_wall_node_invariants():
    """Random pulled populations on a node of the z- wall: the rebuilt populations carry
    rho = sum_{c_z = 0} f + 2 sum_{c_z < 0} f, zero momentum and the non-equilibrium
    stress of the bounce-back-completed set; on an edge (x- and z- walls) the momentum is
    still zero."""
    rng = np.random.default_rng(0)
    W = cmr.equilibrium(torch.ones(1, dtype=torch.float64), torch.zeros(1, 3, dtype=torch.float64))[0]
    f_in = W[None, :] * (1.0 + 0.1 * torch.as_tensor(rng.standard_normal((1, 27))))
    x = torch.tensor([3]); y = torch.tensor([2]); z = torch.tensor([0])
    out = grid.regularized_wall(f_in, grid.face_unknowns(WALLS_Z, (8, 8, 8), x, y, z))
    cz = cmr.C[:, 2]
    rho = f_in[0, cz == 0].sum() + 2 * f_in[0, cz < 0].sum()
    assert torch.isclose(out[0].sum(), rho, rtol=1e-14)
    assert torch.allclose(out[0] @ cmr.C, torch.zeros(3, dtype=torch.float64), atol=1e-15)
    completed = torch.where(cz > 0, f_in[0, cmr.OPP], f_in[0])
    neq = completed - W * rho
    pi_c = torch.einsum("q,qa,qb->ab", neq, cmr.C, cmr.C)
    pi_o = torch.einsum("q,qa,qb->ab", out[0] - W * rho, cmr.C, cmr.C)
    assert torch.allclose(pi_o, pi_c, atol=1e-15)
    edge = grid.regularized_wall(f_in, grid.face_unknowns((True, False, False, False, True, False),
                                                          (8, 8, 8), torch.tensor([0]), y, z))
    assert torch.allclose(edge[0] @ cmr.C, torch.zeros(3, dtype=torch.float64), atol=1e-15)


def test_surface_voxels_of_solid_cubes():
    """A solid cube of edge e inside a periodic block: its surface voxels are the e^3 - (e-2)^3
    voxels with a fluid neighbour, the (e-2)^3 others are inert."""
    for e in (3, 4):
        fl = np.zeros((10, 10, 10), np.uint8)
        fl[2:2 + e, 3:3 + e, 4:4 + e] = grid.SOLID
        surf = grid.surface_voxels(torch.as_tensor(fl), (True, True, True)).numpy()
        assert surf.sum() == e ** 3 - (e - 2) ** 3
        assert not surf[3:1 + e, 4:2 + e, 5:3 + e].any()
        assert not surf[fl == 0].any()


def _slab_channel(H, nu, g, steps, obstacles):
    """Body-forced channel of H + 1 wall-to-wall nodes: between wall faces (z = 0 and z = H),
    or, on a periodic z axis, between the surfaces (z = 2 and z = H + 2) of an obstacle
    slab of 6 voxels (z = 0, 1, 2 and H + 2, H + 3, H + 4, joined through the wrap)."""
    Z = H + 5 if obstacles else H + 1
    fl = np.zeros((Z, 1, 1), np.uint8)
    if obstacles:
        fl[[0, 1, 2, H + 2, H + 3, H + 4]] = grid.SOLID
    st = grid.init_state(np.ones((Z, 1, 1)), np.zeros((3, Z, 1, 1)), np.zeros((Z, 1, 1)), fl)
    p = grid.Params(nu=nu, periodic=(True, True, obstacles), adaptive=False,
                    body_force=(g, 0.0, 0.0), walls=(False,) * 6 if obstacles else WALLS_Z,
                    obstacle_walls=obstacles)
    for _ in range(steps):
        st = grid.step(st, p)
    return st


def test_channel_between_obstacle_slabs_matches_the_wall_face_channel():
    """With the surface voxels of two obstacle slabs as walls, the nodes from wall to wall
    carry the state of the channel between two wall faces (the inert voxels behind the
    surface only feed unknown populations, which the wall replaces), so the profile has the
    exact curvature -g / nu of the closed form and is zero on the walls."""
    H, nu, g, steps = 8, 0.2, 1e-5, 200
    face = _slab_channel(H, nu, g, steps, False)
    obst = _slab_channel(H, nu, g, steps, True)
    # obstacle layout: z = 0, 1 inert, z = 2 wall ... z = H + 2 wall, z = H + 3, H + 4 inert
    sl = slice(2, H + 3)
    assert torch.allclose(obst.f[:, sl], face.f, atol=1e-15)
    assert torch.allclose(obst.u[:, sl], face.u, atol=1e-15)
    inert = [0, 1, H + 3, H + 4]
    W = cmr.equilibrium(torch.ones(1, dtype=torch.float64), torch.zeros(1, 3, dtype=torch.float64))[0]
    assert torch.allclose(obst.f[:, inert, 0, 0], W[:, None].expand(27, 4), atol=0)
    long = _slab_channel(H, nu, g, int(8 * H * H / nu), True)
    u = long.u[0, sl, 0, 0].numpy()
    d2 = u[3:-1] - 2 * u[2:-2] + u[1:-3]
    assert np.allclose(d2, -g / nu, rtol=1e-6)
    assert abs(u[0]) < 1e-15 and abs(u[-1]) < 1e-15


def test_wall_node_with_unknowns_from_several_directions():
    """The corner voxel of a 2 x 2 x 2 solid block embedded in a larger obstacle: any set of
    unknown populations gives zero momentum, mass (known + bounce-back completed) /
    (1 - sum of w over pairs unknown both ways), and the completed set's stress."""
    rng = np.random.default_rng(3)
    W = cmr.equilibrium(torch.ones(1, dtype=torch.float64), torch.zeros(1, 3, dtype=torch.float64))[0]
    f_in = W[None, :] * (1.0 + 0.1 * torch.as_tensor(rng.standard_normal((1, 27))))
    C = cmr.C
    # unknown: sources in the octant x - c with c_x >= 0, c_y >= 0, c_z >= 0 (not the rest)
    unk = ((C[:, 0] >= 0) & (C[:, 1] >= 0) & (C[:, 2] >= 0)).clone()
    unk[13] = False
    unk[(C[:, 0] == 1) & (C[:, 1] == -1) & (C[:, 2] == 0)] = True     # and one stray pair
    unk[(C[:, 0] == -1) & (C[:, 1] == 1) & (C[:, 2] == 0)] = True
    out = grid.regularized_wall(f_in, unk[None, :])
    opp = unk[cmr.OPP]
    both = unk & opp
    assert both.any() and (unk & ~opp).any()
    rho = (f_in[0, ~unk].sum() + f_in[0, cmr.OPP][unk & ~opp].sum()) / (1.0 - W[both].sum())
    assert torch.isclose(out[0].sum(), rho, rtol=1e-14)
    assert torch.allclose(out[0] @ C, torch.zeros(3, dtype=torch.float64), atol=1e-15)
    completed = torch.where(unk & ~opp, f_in[0, cmr.OPP], f_in[0])
    completed = torch.where(both, W * rho, completed)
    pi_c = torch.einsum("q,qa,qb->ab", completed - W * rho, C, C)
    pi_o = torch.einsum("q,qa,qb->ab", out[0] - W * rho, C, C)
    assert torch.allclose(pi_o, pi_c, atol=1e-15)


def test_plate_one_voxel_thick_is_a_wall_at_rest():
    """A plate one voxel thick has no inner voxels, so nothing reaches its voxels from inside
    the obstacle; they are still wall nodes at rest (zero velocity to rounding, every step)
    while the flow around the plate moves."""
    Z, Y, X = 10, 8, 12
    fl = np.zeros((Z, Y, X), np.uint8)
    fl[2:8, 2:6, 6] = grid.SOLID                      # a plate normal to x
    rng = np.random.default_rng(5)
    u0 = np.zeros((3, Z, Y, X))
    u0[0] = 0.05 + 0.01 * rng.standard_normal((Z, Y, X))
    st = grid.init_state(np.ones((Z, Y, X)), u0, np.zeros((Z, Y, X)), fl)
    assert grid.surface_voxels(st.flags, (True, True, True)).sum() == 24
    p = grid.Params(nu=0.02, periodic=(True, True, True), obstacle_walls=True)
    for _ in range(4):
        st = grid.step(st, p)
        plate = st.u[:, 2:8, 2:6, 6]
        assert float(plate.abs().max()) < 1e-15
    assert float(st.u[0].abs().max()) > 0.01
