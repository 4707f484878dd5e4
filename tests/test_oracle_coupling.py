"""Pins of the continuous-scale coupling oracle (Sec. 3.2, 4.2, Algorithm 1)."""
import math

import numpy as np
import pytest
import torch

import synth
from oracle import cmr, coupling, grid

DT = torch.float64
W_BY_NORM = {0: 8.0 / 27.0, 1: 2.0 / 27.0, 2: 1.0 / 54.0, 3: 1.0 / 216.0}


def _w():
    return torch.tensor([W_BY_NORM[int((cmr.C[i] ** 2).sum())] for i in range(27)], dtype=DT)


def _feq(rho, u):
    w = _w()
    cu = u @ cmr.C.T
    return w * rho[..., None] * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * (u * u).sum(-1, keepdim=True))


def _blk(h, nu0=1e-3):
    b = synth._empty_block((6, 6, 6), h=h)
    st = grid.init_state(b.rho0, b.u0, b.c0, b.flags)
    return coupling.Blk(origin=np.zeros(3), h=h, dims=(6, 6, 6), state=st,
                        params=grid.Params(nu=nu0 / h))


def _rand_f(n, seed):
    g = torch.Generator().manual_seed(seed)
    rho = 1 + 0.02 * (2 * torch.rand(n, generator=g, dtype=DT) - 1)
    u = 0.08 * (2 * torch.rand(n, 3, generator=g, dtype=DT) - 1)
    return _feq(rho, u) * (1 + 0.05 * (2 * torch.rand(n, 27, generator=g, dtype=DT) - 1))


def test_k_hat_is_identity_for_equal_scales_and_mapping_keeps_rho_u():
    a, b = _blk(1.0), _blk(1.0)
    K = coupling.k_hat(a, b)
    assert torch.allclose(K, torch.ones(27, dtype=DT), rtol=0, atol=1e-15)
    f = _rand_f(64, 1)
    assert torch.allclose(coupling.map_populations(f, K), f, rtol=0, atol=1e-15)
    K2 = coupling.k_hat(_blk(1.0), _blk(1 / 1.5))
    fm = coupling.map_populations(f, K2)
    r0, u0 = cmr.macros(f)
    r1, u1 = cmr.macros(fm)
    assert torch.allclose(r0, r1, atol=1e-15, rtol=0) and torch.allclose(u0, u1, atol=1e-15, rtol=0)


@pytest.mark.parametrize("hc,hf", [(1.0, 0.5), (1.0, 1 / 1.5), (1 / 1.5, 1 / 2.25)])
def test_mapping_round_trip_is_identity(hc, hf):
    c, f_ = _blk(hc), _blk(hf)
    f = _rand_f(64, 2)
    there = coupling.map_populations(f, coupling.k_hat(c, f_))
    back = coupling.map_populations(there, coupling.k_hat(f_, c))
    assert torch.allclose(back, f, rtol=0, atol=2e-15)


@pytest.mark.parametrize("hc,hf", [(1.0, 0.5), (1.0, 1 / 1.5), (1 / 1.5, 1 / 2.25)])
def test_mapping_rescales_chapman_enskog_stress(hc, hf):
    """Sec. 4.2.1: the first-order non-equilibrium part eps f^(1) = w/(2 cs^4) Q : Pi^(1)
    with Pi^(1) = -2 cs^2 rho S_hat / S.  A post-collision coarse state f^eq + (1 - S_c)
    eps f^(1)_c, with the strain rate S_hat in coarse lattice units, must map onto the fine
    post-collision state built with S_hat_f = S_hat_c * dx_f / dx_c and S_f."""
    cb, fb = _blk(hc), _blk(hf)
    Sc = coupling.shear_rate(cb.params.nu)
    Sf = coupling.shear_rate(fb.params.nu)
    cs2 = 1.0 / 3.0
    g = torch.Generator().manual_seed(3)
    n = 16
    rho = 1 + 0.01 * torch.rand(n, generator=g, dtype=DT)
    u = 0.05 * (2 * torch.rand(n, 3, generator=g, dtype=DT) - 1)
    A = 1e-3 * (2 * torch.rand(n, 3, 3, generator=g, dtype=DT) - 1)
    shat = 0.5 * (A + A.transpose(-1, -2))
    shat = shat - torch.eye(3, dtype=DT) * (shat.diagonal(dim1=-2, dim2=-1).sum(-1) / 3)[:, None, None]
    Q = cmr.C[:, :, None] * cmr.C[:, None, :] - cs2 * torch.eye(3, dtype=DT)

    def post_collision(S, strain):
        Pi = -2 * cs2 * rho[:, None, None] * strain / S
        f1 = _w() / (2 * cs2 * cs2) * torch.einsum("qab,nab->nq", Q, Pi)
        return _feq(rho, u) + (1 - S) * f1

    coarse = post_collision(Sc, shat)
    fine_expected = post_collision(Sf, shat * (hf / hc))
    mapped = coupling.map_populations(coarse, coupling.k_hat(cb, fb))
    # the second-order (stress) content must agree; compare the central second moments
    def stress(f):
        r, uu = cmr.macros(f)
        cb_ = cmr.C - uu[:, None, :]
        return torch.einsum("nqa,nqb,nq->nab", cb_, cb_, f)
    assert torch.allclose(stress(mapped), stress(fine_expected), rtol=0, atol=1e-14)


def test_trilinear_interpolation_exact_on_affine_data_and_drops_solids():
    b = synth._empty_block((7, 6, 5), origin=(2.0, 3.0, 1.0), h=0.75)
    st = grid.init_state(b.rho0, b.u0, b.c0, b.flags)
    blk = coupling.Blk(origin=np.array(b.origin), h=0.75, dims=b.dims, state=st,
                       params=grid.Params(nu=0.01))
    xs, ys, zs = b.node_coords()
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    lin = torch.as_tensor(0.1 + 0.02 * X - 0.03 * Y + 0.05 * Z)
    fsrc = lin[None].repeat(27, 1, 1, 1)
    g = torch.Generator().manual_seed(4)
    pos = torch.stack([2.0 + 4.5 * torch.rand(40, generator=g, dtype=DT),
                       3.0 + 3.75 * torch.rand(40, generator=g, dtype=DT),
                       1.0 + 3.0 * torch.rand(40, generator=g, dtype=DT)], -1)
    f, c, ok = coupling.interpolate(blk, fsrc, lin, pos)
    want = 0.1 + 0.02 * pos[:, 0] - 0.03 * pos[:, 1] + 0.05 * pos[:, 2]
    assert ok.all()
    assert torch.allclose(c, want, atol=1e-15, rtol=0)
    assert torch.allclose(f[:, 5], want, atol=1e-15, rtol=0)
    # a solid corner is dropped: with every node solid except one, the result is that node
    flags = torch.full_like(st.flags, synth.SOLID)
    flags[1, 1, 1] = 0
    blk.state.flags = flags
    p = torch.tensor([[2.0 + 0.75 * 1.4, 3.0 + 0.75 * 1.2, 1.0 + 0.75 * 1.7]], dtype=DT)
    f, c, ok = coupling.interpolate(blk, fsrc, lin, p)
    assert ok.all() and c.item() == pytest.approx(lin[1, 1, 1].item(), abs=1e-15)
    blk.state.flags = torch.full_like(st.flags, synth.SOLID)
    _, _, ok = coupling.interpolate(blk, fsrc, lin, p)
    assert not ok.any()


def test_temporal_lagrange_exact_on_quadratics():
    for h in (1 / 1.5, 1 / 2.25, 0.3):
        l = math.ceil(1 / h - 1e-9)
        t0, t1, t2 = 0.0, (l - 1) * h, l * h
        L = coupling.MultiScale.lagrange3(t0, t1, t2, 1.0)
        for (a, b_, c) in [(0.3, -1.2, 2.0), (1.0, 0.0, 0.0), (0.0, 1.0, 0.0)]:
            q = lambda t: a + b_ * t + c * t * t
            assert sum(Li * q(ti) for Li, ti in zip(L, (t0, t1, t2))) == pytest.approx(q(1.0), abs=1e-14)


def test_substep_counts_follow_the_paper():
    sc = synth.multiscale(scale=0.125)
    ms = coupling.MultiScale.build(sc)
    assert [b.substeps for b in ms.blocks] == [1, 2, 3]      # floor(1.5)+1, floor(2.25)+1
    assert [b.integer_ratio for b in ms.blocks] == [True, False, False]
    assert [b.parent for b in ms.blocks[1:]] == [0, 1]
    assert ms.blocks[1].params.nu == pytest.approx(sc.nu * 1.5)
    assert ms.blocks[2].params.nu == pytest.approx(sc.nu * 2.25)


def _uniform_scene(hs, origins, dims, u=(0.06, -0.02, 0.03)):
    blocks = []
    for h, o, d in zip(hs, origins, dims):
        b = synth._empty_block(d, origin=o, h=h)
        b.u0[0], b.u0[1], b.u0[2] = u
        blocks.append(b)
    return synth.Scene(blocks=blocks, periodic=(True, True, True), nu=0.01)


@pytest.mark.parametrize("ratios", [(2.0,), (1.5, 2.25)])
def test_uniform_flow_stays_uniform_across_blocks(ratios):
    """A uniform equilibrium flow is a fixed point of every step, mapping and interpolation,
    for integer and non-integer spacing ratios."""
    hs = [1.0] + [1.0 / r for r in ratios]
    origins = [(0, 0, 0), (3.0, 2.5, 3.25), (4.0, 3.5, 4.0)][: len(hs)]
    dims = [(14, 12, 12), (12, 12, 11), (8, 9, 8)][: len(hs)]
    ms = coupling.MultiScale.build(_uniform_scene(hs, origins, dims), f32_inputs=False)
    f_ref = [b.state.f.clone() for b in ms.blocks]
    ms.run(3)
    for b, fr in zip(ms.blocks, f_ref):
        assert torch.allclose(b.state.f, fr, rtol=0, atol=1e-14)


def test_integer_ratio_block_tracks_the_coarse_flow():
    """alpha = 2 multi-block case (the Fig. 5 comparison shape) on a Taylor-Green vortex:
    the refined block's velocity stays close to the coarse solution at the same points."""
    sc = synth.taylor_green(16, nz=4, re=50)
    b1 = synth._empty_block((12, 12, 6), origin=(4.0, 4.0, 0.5), h=0.5)
    k = 2 * math.pi / 16
    xs, ys, zs = b1.node_coords()
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    b1.u0[0] = 0.05 * np.sin(k * X) * np.cos(k * Y)
    b1.u0[1] = -0.05 * np.cos(k * X) * np.sin(k * Y)
    sc.blocks.append(b1)
    ms = coupling.MultiScale.build(sc, f32_inputs=False)
    assert ms.blocks[1].substeps == 2 and ms.blocks[1].integer_ratio
    ms.run(2)
    for b in ms.blocks:
        assert torch.isfinite(b.state.f).all()
    fine = ms.blocks[1]
    z, y, x = torch.nonzero((fine.state.flags & synth.GHOST) == 0, as_tuple=True)
    pos = coupling.node_positions(fine, z, y, x)
    coarse = ms.blocks[0]
    u_c = torch.stack([coupling.interpolate(coarse, coarse.state.u[a][None].repeat(27, 1, 1, 1),
                                            coarse.state.u[a], pos)[1] for a in range(3)], -1)
    diff = (fine.state.u[:, z, y, x].T - u_c).abs().max().item()
    # the trilinear interpolation of the coarse field alone differs by ~2e-3 at 16 nodes
    # per wavelength; two coupled steps must stay within twice that
    assert diff < 0.1 * 0.05


def test_scale_boundary_node_inside_a_coarse_obstacle_takes_the_rest_state():
    """A ghost node whose 8 source corners are all obstacle voxels cannot be interpolated;
    it holds the rest state (rho = 1, u = 0, scalar 0) after every mapping."""
    sc = synth.random_scene(dims=(12, 12, 12), seed=5, periodic=(False, False, False), nu=0.01)
    b0 = sc.blocks[0]
    b0.flags[:] = 0
    b0.flags[2:8, 2:8, 2:8] = synth.SOLID            # coarse obstacle cube, nodes 2..7
    fine = synth._empty_block((10, 10, 10), origin=(3.0, 3.0, 3.0), h=0.5)
    fine.u0[0] = 0.02
    fine.c0[:] = 0.7
    sc.blocks.append(fine)
    ms = coupling.MultiScale.build(sc)
    ms.step()
    b = ms.blocks[1]
    ghost = (b.state.flags & coupling.GHOST) != 0
    pos = [3.0 + 0.5 * np.arange(10)] * 3
    z, y, x = np.meshgrid(*reversed(pos), indexing="ij")
    inside = (x >= 2) & (x + 1 <= 7) & (y >= 2) & (y + 1 <= 7) & (z >= 2) & (z + 1 <= 7)
    sel = torch.as_tensor(inside) & ghost
    assert int(sel.sum()) > 0
    feq = cmr.equilibrium(torch.ones(1, dtype=torch.float64), torch.zeros(1, 3, dtype=torch.float64))[0]
    assert torch.allclose(b.state.f[:, sel], feq[:, None].expand(27, int(sel.sum())), atol=1e-15)
    assert (b.state.u[:, sel] == 0).all() and (b.state.c[sel] == 0).all()
