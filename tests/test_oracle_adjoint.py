"""Pin of the FP64 adjoint oracle: reverse-mode gradients of the smoke-control loss agree
with central finite differences of the same FP64 forward model."""
import numpy as np
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
