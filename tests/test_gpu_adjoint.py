"""Hand-written GPU adjoint of collide-stream + scalar advection (with checkpointing) against
the FP64 adjoint oracle and against finite differences.

Tolerance: the FP32 adjoint's gradient must match the FP64 gradient to 1e-3 in relative L2
norm (FP32 rounding of forward and reverse accumulates over the horizon; 1e-3 leaves an
order of magnitude of margin on the short horizons here)."""
import numpy as np
import pytest
import torch

import synth
from oracle import adjoint as oadj
from oracle import grid
from tests.helpers import f32

pytestmark = pytest.mark.gpu


def _domain(sc, storage="fp32"):
    from paper_1807_02284_gb300 import lbm
    b = sc.blocks[0]
    dom = lbm.Domain(b.dims, sc.nu, periodic=sc.periodic, adaptive=sc.adaptive, storage=storage)
    dom.set_flags(b.flags)
    return dom


def gpu_grad(sc, target, steps, every, storage="fp32"):
    """(L, dL/du0, c_T) from the GPU forward + hand-written adjoint."""
    from paper_1807_02284_gb300 import lbm
    b = sc.blocks[0]
    dom = _domain(sc, storage)
    dom.init_macro(f32(b.u0), rho=f32(b.rho0), c=f32(b.c0))
    dom.set_tape(every)
    dom.step(steps)
    c = dom.read_field(lbm.LBM_FIELD_SCALAR, lbm.LBM_F64)
    resid = c - target.reshape(-1)
    L = 0.5 * float((resid ** 2).sum())
    dLdc = torch.tensor(resid, dtype=torch.float32, device="cuda")
    g = torch.empty(3 * b.flags.size, dtype=torch.float32, device="cuda")
    dom.adjoint_step(steps, dLdc, g)
    dom.sync()
    dom.close()
    return L, g.cpu().numpy().astype(np.float64).reshape(b.u0.shape), c


def oracle_grad(sc, target, steps):
    b = sc.blocks[0]
    p = grid.Params(nu=sc.nu, periodic=sc.periodic, adaptive=sc.adaptive)
    return oadj.loss_and_grad(f32(b.u0).astype(np.float64), f32(b.rho0).astype(np.float64),
                              f32(b.c0).astype(np.float64), b.flags, p, steps, target)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("n,steps,every,sphere", [(12, 8, 3, False), (16, 20, 5, False),
                                                  (14, 12, 4, True)])
def test_adjoint_matches_fp64_oracle(lib, n, steps, every, sphere):
    sc, target = synth.adjoint_scene(n=n, seed=5, nu=0.01, amp=0.05)
    if sphere:
        synth.voxelise_spheres(sc.blocks[0], [(n / 2 + 1.5, n / 2, n / 2 - 1, 2.5)])
    Lg, gg, cg = gpu_grad(sc, target, steps, every)
    Lo, go, co = oracle_grad(sc, target, steps)
    e = rel(gg, go.numpy())
    print(f"adjoint n={n} steps={steps} k={every} sphere={sphere}: L gpu {Lg:.6e} oracle {Lo:.6e}, "
          f"rel L2 grad err {e:.2e}")
    assert abs(Lg - Lo) <= 1e-4 * abs(Lo)
    assert e <= 1e-3


def gpu_grad_velocity_loss(sc, u_target, steps, every, storage="fp32"):
    """(L, dL/du0) for L = 1/2 sum |u_T - u_target|^2 (no scalar term: dL/dc_T = 0)."""
    from paper_1807_02284_gb300 import lbm
    b = sc.blocks[0]
    dom = _domain(sc, storage)
    dom.init_macro(f32(b.u0), rho=f32(b.rho0), c=f32(b.c0))
    dom.set_tape(every)
    dom.step(steps)
    u = dom.read_field(lbm.LBM_FIELD_U, lbm.LBM_F64)
    resid = u - u_target.reshape(-1)
    L = 0.5 * float((resid ** 2).sum())
    dLdu = torch.tensor(resid, dtype=torch.float32, device="cuda")
    dLdc = torch.zeros(b.flags.size, dtype=torch.float32, device="cuda")
    g = torch.empty(3 * b.flags.size, dtype=torch.float32, device="cuda")
    dom.adjoint_step(steps, dLdc, g, dL_du=dLdu)
    dom.sync()
    dom.close()
    return L, g.cpu().numpy().astype(np.float64).reshape(b.u0.shape)


@pytest.mark.parametrize("sphere", [False, True])
def test_adjoint_fp16_storage_matches_fp64_oracle(lib, sphere):
    """FP16-shifted storage: checkpoints widen the stored deviations exactly to FP32 and
    each segment is replayed and reversed in FP32 from them, so the gradient is that of the
    trajectory through the rounded checkpoints.  The reference is the FP64 oracle's gradient
    along the same kind of trajectory: deviations rounded to binary16 after every forward
    step, segments replayed from the rounded states, the rounding passed through as the
    identity.  Bounds: 2e-3 of the loss (the FP16 forward's own bound), and 1e-3 relative L2
    for the gradient (FP32 against FP64 arithmetic along one trajectory, as for FP32 storage,
    plus the rare deviation that rounds differently from FP32 and FP64 values).

    With the obstacle the loss is on the final velocity only.  The scalar's semi-Lagrangian
    sample has a kink wherever a velocity component is zero (the departure cell changes
    side), and FP16 storage makes exact cancellations of a node's momentum likely next to a
    bounce-back wall: there the one-sided derivative the GPU takes depends on the sign of
    FP32 rounding noise.  A velocity loss has no scalar adjoint (dL/dc = 0) and so no such
    kink; the scalar's adjoint under FP16 storage is covered by the case without obstacle."""
    n, steps, every = 14, 12, 4
    sc, target = synth.adjoint_scene(n=n, seed=5, nu=0.01, amp=0.05)
    if sphere:
        synth.voxelise_spheres(sc.blocks[0], [(n / 2 + 1.5, n / 2, n / 2 - 1, 2.5)])
    b = sc.blocks[0]
    p = grid.Params(nu=sc.nu, periodic=sc.periodic, adaptive=sc.adaptive)
    args = (f32(b.u0).astype(np.float64), f32(b.rho0).astype(np.float64),
            f32(b.c0).astype(np.float64), b.flags, p, steps)
    ck = oadj.fp16_storage_checkpoints(*args, every)
    if sphere:
        u_target = synth.random_velocity(b.shape_zyx, 77, amp=0.05)
        u0 = torch.as_tensor(args[0])
        with torch.no_grad():
            # the scalar term of the oracle's loss vanishes with its own final scalar as target
            c_fin = oadj.forward(u0, *args[1:], use_checkpoint=False, restart=ck).c
            c_plain = oadj.forward(u0, *args[1:], use_checkpoint=False).c
        Lg, gg = gpu_grad_velocity_loss(sc, u_target, steps, every, storage="fp16")
        Lo, go, _ = oadj.loss_and_grad(*args, c_fin, u_target=u_target, restart=ck)
        L32, g32 = gpu_grad_velocity_loss(sc, u_target, steps, every)
        _, go32, _ = oadj.loss_and_grad(*args, c_plain, u_target=u_target)
    else:
        Lg, gg, _ = gpu_grad(sc, target, steps, every, storage="fp16")
        Lo, go, _ = oadj.loss_and_grad(*args, target, restart=ck)
        L32, g32, _ = gpu_grad(sc, target, steps, every)
        _, go32, _ = oracle_grad(sc, target, steps)
    e, e32 = rel(gg, go.numpy()), rel(g32, go32.numpy())
    print(f"adjoint fp16 sphere={sphere}: L {Lg:.6e} oracle {Lo:.6e}, rel L2 grad err {e:.2e} "
          f"(fp32 storage against the plain oracle {e32:.2e})")
    assert abs(Lg - Lo) <= 2e-3 * abs(Lo)
    assert e <= 1e-3
    assert e32 <= 1e-3


def test_adjoint_fixed_rates_matches_fp64_oracle(lib):
    """Fixed high-order rates (adaptive factor off, phi = 1): no gradient flows through the
    lagged velocity field, only through populations and the scalar."""
    sc, target = synth.adjoint_scene(n=12, seed=6, nu=0.01, amp=0.05)
    sc.adaptive = False
    Lg, gg, _ = gpu_grad(sc, target, 10, 4)
    Lo, go, _ = oracle_grad(sc, target, 10)
    e = rel(gg, go.numpy())
    print(f"adjoint fixed rates: rel L2 grad err {e:.2e}")
    assert abs(Lg - Lo) <= 1e-4 * abs(Lo)
    assert e <= 1e-3


@pytest.mark.parametrize("scalar_source", [False, True])
def test_inflow_velocity_gradient_matches_fp64_oracle(lib, scalar_source):
    """Inflow disk on the x = 0 plane of the periodic box (velocity carried unchanged from
    step to step): dL/du0 everywhere against the FP64 oracle, dL/d(inflow) equal to dL/du0 at
    the inflow nodes and 0 elsewhere."""
    from paper_1807_02284_gb300 import lbm
    n, steps, every = 12, 10, 4
    sc, target = synth.adjoint_scene(n=n, seed=11, nu=0.01, amp=0.05)
    b = sc.blocks[0]
    rng = np.random.default_rng(3)
    zi, yi, _ = synth.inflow_disk(b, (6, 6), 3.0, 0.05, rng=rng, noise=0.2, scalar=scalar_source)
    dom = _domain(sc)
    dom.init_macro(f32(b.u0), rho=f32(b.rho0), c=f32(b.c0))
    dom.set_tape(every)
    dom.step(steps)
    c = dom.read_field(lbm.LBM_FIELD_SCALAR, lbm.LBM_F64)
    dLdc = torch.tensor(c - target.reshape(-1), dtype=torch.float32, device="cuda")
    g = torch.empty(3 * b.flags.size, dtype=torch.float32, device="cuda")
    gi = torch.full_like(g, 7.0)
    dom.adjoint_step(steps, dLdc, g, dL_dinflow=gi)
    dom.sync()
    dom.close()
    gg = g.cpu().numpy().astype(np.float64).reshape(b.u0.shape)
    gin = gi.cpu().numpy().astype(np.float64).reshape(b.u0.shape)
    _, go, _ = oracle_grad(sc, target, steps)
    e = rel(gg, go.numpy())
    ein = rel(gg[:, zi, yi, 0], go.numpy()[:, zi, yi, 0])
    print(f"inflow gradient (scalar source {scalar_source}): rel L2 all {e:.2e}, inflow nodes {ein:.2e}")
    assert e <= 1e-3 and ein <= 1e-3
    mask = np.zeros(b.flags.shape, bool)
    mask[zi, yi, 0] = True
    assert np.array_equal(gin[:, mask], gg[:, mask]) and (gin[:, ~mask] == 0).all()


def _open_face_grad(n, steps, every, plume, periodic=(False, False, False), seed=13):
    from paper_1807_02284_gb300 import lbm
    sc, target = synth.adjoint_scene(n=n, seed=seed, nu=0.01, amp=0.05)
    sc.periodic = periodic
    b = sc.blocks[0]
    if plume:
        rng = np.random.default_rng(4)
        synth.inflow_disk(b, (n / 2, n / 2), n / 4, 0.05, rng=rng, noise=0.2, scalar=True)
        synth.voxelise_spheres(b, [(0.6 * n, n / 2, 0.55 * n, 0.15 * n)])
    dom = _domain(sc)
    dom.init_macro(f32(b.u0), rho=f32(b.rho0), c=f32(b.c0))
    dom.set_tape(every)
    dom.step(steps)
    c = dom.read_field(lbm.LBM_FIELD_SCALAR, lbm.LBM_F64)
    dLdc = torch.tensor(c - target.reshape(-1), dtype=torch.float32, device="cuda")
    g = torch.empty(3 * b.flags.size, dtype=torch.float32, device="cuda")
    dom.adjoint_step(steps, dLdc, g)
    dom.sync()
    dom.close()
    return g.cpu().numpy()


def test_open_face_gradients_are_bit_reproducible(lib):
    """Clamped pulls on open faces are summed in a fixed order (no atomics): two runs of the
    same 40^3 plume-like scene (inflow disk with a scalar source on x = 0, an obstacle) give
    bit-identical gradients, with every face open and with one periodic axis."""
    for periodic in ((False, False, False), (False, True, False)):
        g1 = _open_face_grad(40, 12, 4, True, periodic)
        g2 = _open_face_grad(40, 12, 4, True, periodic)
        assert np.abs(g1).max() > 0
        assert np.array_equal(g1.view(np.uint32), g2.view(np.uint32)), periodic


@pytest.mark.parametrize("periodic", [(True, False, False), (False, True, True)])
def test_mixed_open_and_periodic_faces_adjoint_matches_fp64_oracle(lib, periodic):
    """Open faces on some axes only: the clamped pulls are filed under their lowest clamped
    axis, which a periodic axis never is."""
    n, steps = 12, 8
    sc, target = synth.adjoint_scene(n=n, seed=17, nu=0.01, amp=0.05)
    sc.periodic = periodic
    gg = _open_face_grad(n, steps, 3, False, periodic, seed=17).astype(np.float64)
    _, go, _ = oracle_grad(sc, target, steps)
    e = rel(gg.reshape(go.shape), go.numpy())
    print(f"periodic {periodic}: rel L2 {e:.2e}")
    assert e <= 1e-3


@pytest.mark.parametrize("plume", [False, True])
def test_open_faces_adjoint_matches_fp64_oracle(lib, plume):
    """Open (zero-gradient) faces: a face node's populations are pulled more than once, its
    velocity enters its own clamped difference, and its scalar sample can clamp.  With
    plume=True: inflow disk with a scalar source on the x = 0 face and an obstacle, as in the
    smoke scenes."""
    from paper_1807_02284_gb300 import lbm
    n, steps, every = 12, 10, 3
    sc, target = synth.adjoint_scene(n=n, seed=13, nu=0.01, amp=0.05)
    sc.periodic = (False, False, False)
    b = sc.blocks[0]
    zi = yi = None
    if plume:
        rng = np.random.default_rng(4)
        zi, yi, _ = synth.inflow_disk(b, (6, 6), 3.0, 0.05, rng=rng, noise=0.2, scalar=True)
        synth.voxelise_spheres(b, [(7.5, 6.0, 6.5, 1.8)])
    dom = _domain(sc)
    dom.init_macro(f32(b.u0), rho=f32(b.rho0), c=f32(b.c0))
    dom.set_tape(every)
    dom.step(steps)
    c = dom.read_field(lbm.LBM_FIELD_SCALAR, lbm.LBM_F64)
    dLdc = torch.tensor(c - target.reshape(-1), dtype=torch.float32, device="cuda")
    g = torch.empty(3 * b.flags.size, dtype=torch.float32, device="cuda")
    dom.adjoint_step(steps, dLdc, g)
    dom.sync()
    dom.close()
    gg = g.cpu().numpy().astype(np.float64).reshape(b.u0.shape)
    _, go, _ = oracle_grad(sc, target, steps)
    go = go.numpy()
    e = rel(gg, go)
    face = np.zeros(b.flags.shape, bool)
    face[0], face[-1], face[:, 0], face[:, -1], face[:, :, 0], face[:, :, -1] = (True,) * 6
    ef = rel(gg[:, face], go[:, face])
    print(f"open faces (plume {plume}): rel L2 all {e:.2e}, face nodes {ef:.2e}")
    assert e <= 1e-3 and ef <= 1e-3


@pytest.mark.parametrize("kind", ["faces", "obstacles", "both"])
def test_adjoint_with_walls_matches_fp64_oracle(lib, kind):
    """No-slip walls (the Sec. 6.1 regularized wall): wall faces (floor and lid), obstacle
    surfaces as walls (a sphere and a plate one voxel thick), or both; the transpose of the
    wall completion and rebuild against the FP64 oracle's gradient."""
    import dataclasses
    from paper_1807_02284_gb300 import lbm
    n, steps, every = 12, 10, 3
    sc, target = synth.adjoint_scene(n=n, seed=15, nu=0.01, amp=0.05)
    sc.periodic = (True, True, False)
    b = sc.blocks[0]
    faces = (False,) * 4 + ((True, True) if kind != "obstacles" else (False, False))
    obst = kind != "faces"
    if obst:
        synth.voxelise_spheres(b, [(6.5, 5.5, 6.0, 2.2)])
        b.flags[3:8, 2:5, 10] |= synth.SOLID
        b.rho0[(b.flags & synth.SOLID) != 0] = 1.0
    dom = _domain(sc)
    dom.set_walls(faces, obstacles=obst)
    dom.init_macro(f32(b.u0), rho=f32(b.rho0), c=f32(b.c0))
    dom.set_tape(every)
    dom.step(steps)
    c = dom.read_field(lbm.LBM_FIELD_SCALAR, lbm.LBM_F64)
    dLdc = torch.tensor(c - target.reshape(-1), dtype=torch.float32, device="cuda")
    g = torch.empty(3 * b.flags.size, dtype=torch.float32, device="cuda")
    dom.adjoint_step(steps, dLdc, g)
    dom.sync()
    dom.close()
    gg = g.cpu().numpy().astype(np.float64).reshape(b.u0.shape)
    p = dataclasses.replace(grid.Params(nu=sc.nu, periodic=sc.periodic, adaptive=sc.adaptive),
                            walls=faces, obstacle_walls=obst)
    _, go, _ = oadj.loss_and_grad(f32(b.u0).astype(np.float64), f32(b.rho0).astype(np.float64),
                                  f32(b.c0).astype(np.float64), b.flags, p, steps, target)
    go = go.numpy()
    e = rel(gg, go)
    print(f"walls ({kind}): rel L2 {e:.2e}")
    assert e <= 1e-3


@pytest.mark.parametrize("open_faces", [False, True])
def test_adjoint_local_strain_mode_matches_fp64_oracle(lib, open_faces):
    """The adaptive factor from the node's own strain rate (Sec. 4.2.1 reading): the factor's
    adjoint flows into the node's non-equilibrium moments, rho and u instead of the lagged
    velocity field.  Against the FP64 oracle's gradient."""
    from paper_1807_02284_gb300 import lbm
    n, steps, every = 12, 10, 3
    sc, target = synth.adjoint_scene(n=n, seed=16, nu=0.01, amp=0.06)
    if open_faces:
        sc.periodic = (False, False, False)
        synth.voxelise_spheres(sc.blocks[0], [(6.5, 5.5, 6.0, 2.0)])
    b = sc.blocks[0]
    b.rho0[(b.flags & synth.SOLID) != 0] = 1.0
    dom = lbm.Domain(b.dims, sc.nu, periodic=sc.periodic, adaptive=sc.adaptive, grad_mode="local")
    dom.set_flags(b.flags)
    dom.init_macro(f32(b.u0), rho=f32(b.rho0), c=f32(b.c0))
    dom.set_tape(every)
    dom.step(steps)
    c = dom.read_field(lbm.LBM_FIELD_SCALAR, lbm.LBM_F64)
    dLdc = torch.tensor(c - target.reshape(-1), dtype=torch.float32, device="cuda")
    g = torch.empty(3 * b.flags.size, dtype=torch.float32, device="cuda")
    dom.adjoint_step(steps, dLdc, g)
    dom.sync()
    dom.close()
    gg = g.cpu().numpy().astype(np.float64).reshape(b.u0.shape)
    p = grid.Params(nu=sc.nu, periodic=sc.periodic, adaptive=sc.adaptive, grad_mode="local")
    _, go, _ = oadj.loss_and_grad(f32(b.u0).astype(np.float64), f32(b.rho0).astype(np.float64),
                                  f32(b.c0).astype(np.float64), b.flags, p, steps, target)
    e = rel(gg, go.numpy())
    print(f"local strain (open {open_faces}): rel L2 {e:.2e}")
    assert e <= 1e-3


def test_adjoint_config5_copy_32_cubed_200_steps(lib):
    """The smoke-control problem scaled to 32^3 (every length / 4), nu = 1e-3, 200 steps,
    checkpoint every 20: FP32 GPU adjoint against the FP64 oracle gradient."""
    sc, target = synth.adjoint_scene(n=32, seed=5, nu=1e-3, amp=0.05, steps=200)
    Lg, gg, _ = gpu_grad(sc, target, 200, 20)
    Lo, go, _ = oracle_grad(sc, target, 200)
    e = rel(gg, go.numpy())
    print(f"config-5 copy 32^3 x 200: L gpu {Lg:.6e} oracle {Lo:.6e}, rel L2 grad err {e:.2e}")
    assert abs(Lg - Lo) <= 1e-4 * abs(Lo)
    assert e <= 1e-3


def test_adjoint_full_size_finite_difference_along_gradient(lib):
    """128^3 smoke control, 200 steps, checkpoint every 20: the GPU forward's central
    difference along the normalised gradient equals the gradient norm."""
    from paper_1807_02284_gb300 import lbm
    sc, target = synth.adjoint_scene(n=128, seed=5, nu=1e-3, amp=0.05, steps=200)
    b = sc.blocks[0]
    steps = 200
    L0, g, _ = gpu_grad(sc, target, steps, 20)
    gn = float(np.linalg.norm(g))
    vhat = g / gn

    def loss(u):
        dom = _domain(sc)
        dom.init_macro(f32(u), rho=f32(b.rho0), c=f32(b.c0))
        dom.step(steps)
        c = dom.read_field(lbm.LBM_FIELD_SCALAR, lbm.LBM_F64)
        dom.close()
        return 0.5 * float(((c - target.reshape(-1)) ** 2).sum())

    eps = 2e-3
    fd = (loss(b.u0 + eps * vhat) - loss(b.u0 - eps * vhat)) / (2 * eps)
    print(f"128^3 x 200: |dL/du0| = {gn:.6e}, central FD along it = {fd:.6e}")
    assert abs(fd - gn) <= 1e-2 * gn


def test_checkpoint_interval_does_not_change_the_gradient(lib):
    sc, target = synth.adjoint_scene(n=12, seed=6, nu=0.01, amp=0.05)
    _, g1, _ = gpu_grad(sc, target, 9, 1)
    _, g4, _ = gpu_grad(sc, target, 9, 4)
    _, g9, _ = gpu_grad(sc, target, 9, 9)
    assert np.array_equal(g1, g4) and np.array_equal(g1, g9)


def test_adjoint_directional_derivative_matches_central_differences(lib):
    """dL/du0 . v against (L(u0 + e v) - L(u0 - e v)) / 2e of the FP64 forward model."""
    sc, target = synth.adjoint_scene(n=12, seed=9, nu=0.01, amp=0.05)
    b = sc.blocks[0]
    steps = 10
    _, g, _ = gpu_grad(sc, target, steps, 5)
    p = grid.Params(nu=sc.nu, periodic=sc.periodic, adaptive=sc.adaptive)
    rng = np.random.default_rng(3)
    u0 = f32(b.u0).astype(np.float64)
    rho0 = f32(b.rho0).astype(np.float64)
    c0 = f32(b.c0).astype(np.float64)
    for _ in range(2):
        v = rng.standard_normal(b.u0.shape)
        eps = 1e-5
        lp = oadj.loss_only(u0 + eps * v, rho0, c0, b.flags, p, steps, target)
        lm = oadj.loss_only(u0 - eps * v, rho0, c0, b.flags, p, steps, target)
        fd = (lp - lm) / (2 * eps)
        ad = float((g * v).sum())
        print(f"directional derivative: adjoint {ad:.6e}, central FD {fd:.6e}")
        assert abs(ad - fd) <= 2e-3 * abs(fd)


def test_autograd_function_returns_the_adjoint(lib):
    from paper_1807_02284_gb300 import lbm
    from paper_1807_02284_gb300.autograd import smoke_rollout
    sc, target = synth.adjoint_scene(n=12, seed=10, nu=0.01, amp=0.05)
    b = sc.blocks[0]
    dom = _domain(sc)
    u0 = torch.tensor(f32(b.u0), device="cuda", requires_grad=True)
    rho0 = torch.tensor(f32(b.rho0), device="cuda")
    c0 = torch.tensor(f32(b.c0), device="cuda")
    tgt = torch.tensor(f32(target).reshape(-1), device="cuda")
    c = smoke_rollout(u0, dom, 8, 4, rho0, c0)
    loss = 0.5 * ((c - tgt) ** 2).sum()
    loss.backward()
    _, g_ref, _ = gpu_grad(sc, target, 8, 4)
    # dL/dc is formed in float32 here and rounded from float64 in gpu_grad
    assert rel(u0.grad.cpu().numpy().astype(np.float64), g_ref) <= 1e-5
    dom.close()


def test_adjoint_argument_checks(lib):
    from paper_1807_02284_gb300 import lbm
    sc = synth.random_scene(dims=(10, 10, 10), seed=3, periodic=(False, True, True))
    b = sc.blocks[0]
    d = lbm.Domain(b.dims, sc.nu, periodic=sc.periodic, storage="fp16")
    d.init_macro(f32(b.u0))
    d.set_tape(2)                                   # FP16 storage: covered
    d.close()
    d = lbm.Domain(b.dims, sc.nu, periodic=(False, False, False))   # far field: covered
    d.add_scale_block((-4.0, -4.0, -4.0), 2.0, (10, 10, 10))
    d.init_macro(f32(b.u0))
    d.set_tape(2)
    d.close()
    sc, target = synth.adjoint_scene(n=8, seed=1)
    d = _domain(sc)
    b = sc.blocks[0]
    d.init_macro(f32(b.u0))
    g = torch.empty(3 * b.flags.size, device="cuda")
    dc = torch.zeros(b.flags.size, device="cuda")
    with pytest.raises(lbm.LBMError) as ei:
        d.adjoint_step(0, dc, g)
    assert ei.value.status == lbm.LBM_ERR_STATE
    d.set_tape(2)
    d.step(3)
    with pytest.raises(lbm.LBMError) as ei:
        d.adjoint_step(2, dc, g)
    assert ei.value.status == lbm.LBM_ERR_INVALID_ARG
    d.close()
