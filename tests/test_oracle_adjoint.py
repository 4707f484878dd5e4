"""Pin of the FP64 adjoint oracle: reverse-mode gradients of the smoke-control loss agree
with central finite differences of the same FP64 forward model."""
import numpy as np
import pytest
import torch

import synth
from oracle import adjoint, grid


def test_oracle_gradient_matches_central_differences():
    sc, target = synth.adjoint_scene(n=8, seed=7, nu=0.02, amp=0.05)
    b = sc.blocks[0]
    p = grid.Params(nu=sc.nu, periodic=sc.periodic, adaptive=True)
    steps = 6
    L, g, _ = adjoint.loss_and_grad(b.u0, b.rho0, b.c0, b.flags, p, steps, target)
    assert np.isfinite(L) and torch.isfinite(g).all()
    rng = np.random.default_rng(0)
    for _ in range(3):
        v = rng.standard_normal(b.u0.shape)
        eps = 1e-6
        lp = adjoint.loss_only(b.u0 + eps * v, b.rho0, b.c0, b.flags, p, steps, target)
        lm = adjoint.loss_only(b.u0 - eps * v, b.rho0, b.c0, b.flags, p, steps, target)
        fd = (lp - lm) / (2 * eps)
        ad = float((g.numpy() * v).sum())
        assert abs(fd - ad) <= 1e-6 * max(abs(fd), 1e-12) + 1e-13, (fd, ad)


def test_oracle_gradient_with_obstacle_and_velocity_term():
    sc, target = synth.adjoint_scene(n=8, seed=8, nu=0.02, amp=0.05)
    b = sc.blocks[0]
    synth.voxelise_spheres(b, [(4.0, 4.0, 4.0, 1.5)])
    u_target = np.zeros_like(b.u0)
    p = grid.Params(nu=sc.nu, periodic=sc.periodic, adaptive=True)
    steps = 4
    L, g, _ = adjoint.loss_and_grad(b.u0, b.rho0, b.c0, b.flags, p, steps, target, u_target)
    solid = (b.flags & synth.SOLID) != 0
    assert (g.numpy()[:, solid] == 0).all()      # obstacle voxels ignore u0
    v = np.random.default_rng(1).standard_normal(b.u0.shape)
    eps = 1e-6
    lp = adjoint.loss_only(b.u0 + eps * v, b.rho0, b.c0, b.flags, p, steps, target, u_target)
    lm = adjoint.loss_only(b.u0 - eps * v, b.rho0, b.c0, b.flags, p, steps, target, u_target)
    fd = (lp - lm) / (2 * eps)
    assert abs(fd - float((g.numpy() * v).sum())) <= 1e-6 * abs(fd)


def test_oracle_inflow_velocity_gradient_matches_central_differences():
    """Inflow nodes (a disk on the x = 0 plane of a periodic box, velocity carried from step
    to step): the gradient along a perturbation of the inflow velocities alone agrees with
    central differences of the loss."""
    sc, target = synth.adjoint_scene(n=8, seed=9, nu=0.02, amp=0.05)
    b = sc.blocks[0]
    rng = np.random.default_rng(2)
    zi, yi, _ = synth.inflow_disk(b, (4, 4), 2.0, 0.04, rng=rng, noise=0.2, scalar=False)
    p = grid.Params(nu=sc.nu, periodic=sc.periodic, adaptive=True)
    steps = 5
    L, g, _ = adjoint.loss_and_grad(b.u0, b.rho0, b.c0, b.flags, p, steps, target)
    v = np.zeros_like(b.u0)
    v[:, zi, yi, 0] = rng.standard_normal((3, zi.size))
    # the scalar's trilinear sample is piecewise smooth (a kink wherever a departure point
    # crosses a node, i.e. a velocity component passes 0); a small step keeps the
    # difference quotient on one smooth piece
    eps = 1e-7
    lp = adjoint.loss_only(b.u0 + eps * v, b.rho0, b.c0, b.flags, p, steps, target)
    lm = adjoint.loss_only(b.u0 - eps * v, b.rho0, b.c0, b.flags, p, steps, target)
    fd = (lp - lm) / (2 * eps)
    ad = float((g.numpy() * v).sum())
    assert abs(ad) > 1e-9
    assert abs(fd - ad) <= 2e-6 * abs(fd), (fd, ad)


def test_oracle_gradient_on_open_faces_matches_central_differences():
    """Open (zero-gradient) faces with an obstacle: the clamped pulls, clamped velocity
    differences and clamped scalar samples are all inside the differentiated forward model."""
    sc, target = synth.adjoint_scene(n=8, seed=10, nu=0.02, amp=0.05)
    b = sc.blocks[0]
    synth.voxelise_spheres(b, [(4.5, 3.5, 4.0, 1.5)])
    p = grid.Params(nu=sc.nu, periodic=(False, False, False), adaptive=True)
    steps = 5
    L, g, _ = adjoint.loss_and_grad(b.u0, b.rho0, b.c0, b.flags, p, steps, target)
    v = np.random.default_rng(3).standard_normal(b.u0.shape)
    eps = 1e-7
    lp = adjoint.loss_only(b.u0 + eps * v, b.rho0, b.c0, b.flags, p, steps, target)
    lm = adjoint.loss_only(b.u0 - eps * v, b.rho0, b.c0, b.flags, p, steps, target)
    fd = (lp - lm) / (2 * eps)
    ad = float((g.numpy() * v).sum())
    assert abs(fd - ad) <= 2e-6 * abs(fd), (fd, ad)


def test_oracle_multiscale_gradient_matches_central_differences():
    """Two-block continuous-scale domain (h = 1/1.5: sub-cycling, temporal alignment, prior-
    and post-mapping): the gradient of the reference block's final scalar loss with respect
    to both blocks' initial velocities agrees with central differences along a direction."""
    sc = synth.multiscale(seed=2, sphere_seed=3, scale=0.125, flow_amp=0.03, nu=0.004)
    sc.blocks = sc.blocks[:2]
    target = np.zeros(sc.blocks[0].shape_zyx)
    steps = 2
    L, grads, _ = adjoint.ms_loss_and_grad(sc, steps, target)
    rng = np.random.default_rng(4)
    vs = [rng.standard_normal(b.u0.shape) for b in sc.blocks]
    u0 = [np.asarray(b.u0, np.float32).astype(np.float64) for b in sc.blocks]
    eps = 1e-7
    lp = adjoint.ms_loss_only(sc, [u + eps * v for u, v in zip(u0, vs)], steps, target)
    lm = adjoint.ms_loss_only(sc, [u - eps * v for u, v in zip(u0, vs)], steps, target)
    fd = (lp - lm) / (2 * eps)
    ad = sum(float((g.numpy() * v).sum()) for g, v in zip(grads, vs))
    ad1 = float((grads[1].numpy() * vs[1]).sum())
    assert abs(ad1) > 1e-6 * abs(ad)              # the refined block's start matters
    assert abs(fd - ad) <= 2e-6 * abs(fd), (fd, ad)


def test_oracle_farfield_gradient_matches_central_differences():
    """The reference block inside a far-field block (h = 1.5: the far block's aligned step,
    the overlap mapping into it and the boundary mapping out of it): the gradient of the
    reference block's final scalar loss with respect to both blocks' initial velocities
    agrees with central differences along a direction, and the far block's start matters."""
    sc = synth.random_scene(dims=(12, 10, 10), seed=47, periodic=(False, False, False),
                            spheres=[(6.0, 5.0, 5.0, 1.6)], nu=0.01)
    fb = synth.far_block(sc.blocks[0], 1.5, 4.0, seed=6, amp=0.03)
    target = np.zeros(sc.blocks[0].shape_zyx)
    steps = 3
    L, grads, _ = adjoint.ms_loss_and_grad(sc, steps, target, far=(fb,))
    assert len(grads) == 2
    rng = np.random.default_rng(5)
    blocks = list(sc.blocks) + [fb]
    vs = [rng.standard_normal(b.u0.shape) for b in blocks]
    u0 = [np.asarray(b.u0, np.float32).astype(np.float64) for b in blocks]
    eps = 1e-7
    lp = adjoint.ms_loss_only(sc, [u + eps * v for u, v in zip(u0, vs)], steps, target, far=(fb,))
    lm = adjoint.ms_loss_only(sc, [u - eps * v for u, v in zip(u0, vs)], steps, target, far=(fb,))
    fd = (lp - lm) / (2 * eps)
    ad = sum(float((g.numpy() * v).sum()) for g, v in zip(grads, vs))
    ad1 = float((grads[1].numpy() * vs[1]).sum())
    assert abs(ad1) > 1e-6 * abs(ad)              # the far block's start matters
    assert abs(fd - ad) <= 2e-6 * abs(fd), (fd, ad)


@pytest.mark.parametrize("mode", ["local", "walls"])
def test_oracle_gradient_local_strain_and_walls_match_central_differences(mode):
    """The adaptive factor from the node's own strain rate, or no-slip walls (a floor and an
    obstacle with its surface as walls): the forward model the oracle differentiates agrees
    with central differences along a direction."""
    import dataclasses
    sc, target = synth.adjoint_scene(n=8, seed=11, nu=0.02, amp=0.06)
    b = sc.blocks[0]
    if mode == "local":
        p = grid.Params(nu=sc.nu, periodic=(True, True, True), adaptive=True, grad_mode="local")
    else:
        synth.voxelise_spheres(b, [(4.5, 3.5, 4.0, 1.5)])
        b.rho0[(b.flags & synth.SOLID) != 0] = 1.0
        p = dataclasses.replace(grid.Params(nu=sc.nu, periodic=(True, True, False), adaptive=True),
                                walls=(False,) * 4 + (True, False), obstacle_walls=True)
    steps = 5
    L, g, _ = adjoint.loss_and_grad(b.u0, b.rho0, b.c0, b.flags, p, steps, target)
    v = np.random.default_rng(6).standard_normal(b.u0.shape)
    eps = 1e-7
    lp = adjoint.loss_only(b.u0 + eps * v, b.rho0, b.c0, b.flags, p, steps, target)
    lm = adjoint.loss_only(b.u0 - eps * v, b.rho0, b.c0, b.flags, p, steps, target)
    fd = (lp - lm) / (2 * eps)
    ad = float((g.numpy() * v).sum())
    assert abs(ad) > 1e-9
    assert abs(fd - ad) <= 2e-6 * abs(fd), (fd, ad)


def test_binary16_rounding_of_the_shifted_populations():
    """FP16-shifted storage keeps d = f - w in IEEE binary16 (round to nearest, ties to even):
    representable deviations are kept exactly, ties go to the even significand, normal
    values move by at most half an ulp (2^-11 relative), values below the smallest normal
    (2^-14) by at most half the subnormal spacing (2^-25)."""
    from oracle import cmr
    w = cmr.equilibrium(torch.ones(1, dtype=torch.float64), torch.zeros(1, 3, dtype=torch.float64))[0]
    d = torch.tensor([0.0, 2.0 ** -10, -3 * 2.0 ** -12, 1 + 2.0 ** -11, 1 + 3 * 2.0 ** -11,
                      2.0 ** -20, 3 * 2.0 ** -26], dtype=torch.float64)
    want = torch.tensor([0.0, 2.0 ** -10, -3 * 2.0 ** -12, 1.0, 1 + 2.0 ** -9, 2.0 ** -20,
                         2.0 ** -24], dtype=torch.float64)
    f = w[:, None] + d[None, :]
    got = adjoint.round_shifted_to_half(f) - w[:, None]
    # (adding and removing w costs at most an ulp of the sum in float64)
    assert torch.allclose(got, want[None, :].expand(27, -1), rtol=0, atol=2.3e-16)
    g = torch.Generator().manual_seed(3)
    dr = (torch.rand(27, 4096, generator=g, dtype=torch.float64) - 0.5) * 2.0 ** \
        torch.randint(-30, 0, (27, 4096), generator=g).to(torch.float64)
    dr = (w[:, None] + dr) - w[:, None]           # the deviations the populations carry
    err = (adjoint.round_shifted_to_half(w[:, None] + dr) - w[:, None] - dr).abs()
    bound = torch.where(dr.abs() >= 2.0 ** -14, dr.abs() * 2.0 ** -11,
                        torch.full_like(dr, 2.0 ** -25))
    assert bool((err <= bound * (1 + 1e-12) + 1e-16).all())


def test_restart_passes_the_derivative_through():
    """Restarting the forward from states equal to its own keeps loss and gradient exactly;
    restarting from the FP16-storage checkpoints moves the trajectory by the storage
    rounding only (the deviations are small: a few 1e-4 of the populations)."""
    sc, target = synth.adjoint_scene(n=8, seed=7, nu=0.02, amp=0.05)
    b = sc.blocks[0]
    p = grid.Params(nu=sc.nu, periodic=sc.periodic, adaptive=True)
    steps, every = 6, 2
    L, g, _ = adjoint.loss_and_grad(b.u0, b.rho0, b.c0, b.flags, p, steps, target)
    own = {}
    with torch.no_grad():
        st = grid.init_state(b.rho0, b.u0, b.c0, b.flags)
        for n in range(steps):
            if n % every == 0:
                own[n] = (st.f.clone(), st.u.clone(), st.c.clone())
            st = grid.step(st, p)
    L1, g1, _ = adjoint.loss_and_grad(b.u0, b.rho0, b.c0, b.flags, p, steps, target, restart=own)
    assert L1 == L and torch.equal(g1, g)
    ck = adjoint.fp16_storage_checkpoints(b.u0, b.rho0, b.c0, b.flags, p, steps, every)
    assert sorted(ck) == [0, 2, 4]
    for n, (f, u, c) in ck.items():
        fo, uo, co = own[n]
        assert float((f - fo).abs().max()) < 1e-4
        assert float((u - uo).abs().max()) < 1e-4 * 0.05 * 10
    L2, g2, _ = adjoint.loss_and_grad(b.u0, b.rho0, b.c0, b.flags, p, steps, target, restart=ck)
    assert abs(L2 - L) < 1e-3 * abs(L)
    assert float(torch.linalg.norm(g2 - g) / torch.linalg.norm(g)) < 1e-3
