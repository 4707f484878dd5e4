"""Pins of the FP64 oracle against facts fixed outside the oracle itself: the paper's printed
tables (tests/golden), textbook identities, closed-form flows and exact invariants.

Each test is chosen so that a plausible slip in the oracle (a dropped term of M or m^eq, a
wrong sign, a transposed operand, a wrong viscosity relation, a misplaced wall) fails it.
"""
import math
import os

import numpy as np
import pytest
import torch

import synth
from oracle import cmr, grid

DT = torch.float64
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# Textbook D3Q27 lattice weights by |c|^2 (rest, face, edge, corner); Sec. 4.2.1 refers to
# the BGK lattice weights without printing them, so the test writes them down independently
# of the oracle.
W_BY_NORM = {0: 8.0 / 27.0, 1: 2.0 / 27.0, 2: 1.0 / 54.0, 3: 1.0 / 216.0}


def _weights():
    return torch.tensor([W_BY_NORM[int((cmr.C[i] ** 2).sum())] for i in range(27)], dtype=DT)


def _feq_textbook(rho, u):
    """Second-order polynomial equilibrium w_i rho (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u)."""
    w = _weights()
    cu = u @ cmr.C.T
    usq = (u * u).sum(-1, keepdim=True)
    return w * rho[..., None] * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * usq)


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def _rand_state(n, seed):
    g = torch.Generator().manual_seed(seed)
    rho = 1.0 + 0.05 * (2 * torch.rand(n, generator=g, dtype=DT) - 1)
    u = 0.12 * (2 * torch.rand(n, 3, generator=g, dtype=DT) - 1)
    return rho, u


# ----------------------------------------------------------------------------- lattice

def test_velocity_set_matches_printed_list_except_index_13():
    rows = {r[0]: [int(v) for v in r[1:]] for r in _read_golden("paper_velocity_list.txt")}
    printed = torch.tensor([rows["cx"], rows["cy"], rows["cz"]], dtype=DT).T
    diff = (printed != cmr.C).any(dim=1).nonzero().flatten().tolist()
    assert diff == [13]
    assert cmr.C[13].tolist() == [1.0, 0.0, -1.0]
    # the printed list is not a velocity set (duplicate), the read one is all of {-1,0,1}^3
    assert len({tuple(r) for r in printed.tolist()}) == 26
    assert {tuple(int(v) for v in r) for r in cmr.C.tolist()} == {
        (a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)}
    for i in range(27):
        assert torch.equal(cmr.C[cmr.OPP[i]], -cmr.C[i])


def test_printed_m20_makes_moment_matrix_singular_and_reading_does_not():
    rho, u = _rand_state(64, 1)
    M = cmr.moment_matrix(u)
    assert (torch.linalg.matrix_rank(M) == 27).all()
    cb = cmr.C - u[:, None, :]
    printed20 = cb[..., 0] ** 2 * cb[..., 1] * cb[..., 2] ** 2
    Mp = M.clone()
    Mp[..., 20] = printed20
    assert (torch.linalg.matrix_rank(Mp) == 26).all()


def test_moment_matrix_basics_first_row_and_lowest_moments():
    # moments 0..3 of f are rho and sum (c - u) f; 4..6 are the off-diagonal second moments
    rho, u = _rand_state(16, 2)
    g = torch.Generator().manual_seed(3)
    f = torch.rand(16, 27, generator=g, dtype=DT)
    m = (cmr.moment_matrix(u).transpose(-1, -2) @ f[..., None])[..., 0]
    cb = cmr.C - u[:, None, :]
    assert torch.allclose(m[:, 0], f.sum(-1), rtol=0, atol=1e-14)
    for a in range(3):
        assert torch.allclose(m[:, 1 + a], (cb[..., a] * f).sum(-1), rtol=0, atol=1e-14)
    assert torch.allclose(m[:, 4], (cb[..., 0] * cb[..., 1] * f).sum(-1), rtol=0, atol=1e-14)


# ------------------------------------------------------------------------- equilibrium

def test_printed_equilibrium_moments_are_central_moments_of_textbook_equilibrium():
    """M(u)^T f^eq = m^eq for the textbook second-order D3Q27 equilibrium: pins every
    printed m^eq polynomial and every column of M at once."""
    rho, u = _rand_state(4096, 4)
    feq = _feq_textbook(rho, u)
    m = (cmr.moment_matrix(u).transpose(-1, -2) @ feq[..., None])[..., 0]
    assert torch.allclose(m, cmr.m_eq(rho, u), rtol=0, atol=2e-15)


def test_equilibrium_state_is_textbook_polynomial():
    rho, u = _rand_state(512, 5)
    assert torch.allclose(cmr.equilibrium(rho, u), _feq_textbook(rho, u), rtol=0, atol=1e-15)


def test_relaxation_table_matches_paper():
    rows = _read_golden("paper_relaxation.txt")
    S = cmr.relaxation_rates(0.01)
    for r in rows:
        if r[0] == "nu_hi":
            lo, hi, nup = int(r[1]), int(r[2]), float(r[3])
            for i in range(lo, hi + 1):
                assert S[i].item() == pytest.approx(1.0 / (3 * nup + 0.5), rel=1e-15)
        elif r[0] == "a":
            assert cmr.A_DEFAULT == float(r[1])
        elif r[0] == "b":
            assert cmr.B_DEFAULT == float(r[1])
        elif r[0] == "g_max_lo":
            assert cmr.G_MAX_DEFAULT >= float(r[1])
        elif r[0] == "g_max_hi":
            assert cmr.G_MAX_DEFAULT <= float(r[1])
        elif r[0] == "s_conserved":
            assert (S[:4] == float(r[1])).all()
    assert (S[4:9] == 1.0 / (3 * 0.01 + 0.5)).all()


# --------------------------------------------------------------------------- collision

def test_collision_reduces_to_bgk_when_all_rates_equal():
    """With S_i = omega for every moment the CMR collision is the BGK collision
    f - omega (f - f^eq) with the textbook equilibrium."""
    rho, u = _rand_state(256, 6)
    g = torch.Generator().manual_seed(7)
    f = _feq_textbook(rho, u) * (1 + 0.05 * (2 * torch.rand(256, 27, generator=g, dtype=DT) - 1))
    for omega in (0.7, 1.0, 1.6):
        S = torch.full((27,), omega, dtype=DT)
        post, r, uu = cmr.collide(f, S)
        rho_f = f.sum(-1)
        u_f = (f @ cmr.C) / rho_f[:, None]
        bgk = f - omega * (f - _feq_textbook(rho_f, u_f))
        assert torch.allclose(post, bgk, rtol=0, atol=1e-15)


def test_collision_conserves_mass_and_momentum_and_fixes_equilibrium():
    rho, u = _rand_state(256, 8)
    g = torch.Generator().manual_seed(9)
    f = _feq_textbook(rho, u) * (1 + 0.1 * (2 * torch.rand(256, 27, generator=g, dtype=DT) - 1))
    S = cmr.relaxation_rates(1e-3, phi=torch.rand(256, generator=g, dtype=DT) * 4 + 1)
    post, _, _ = cmr.collide(f, S)
    assert torch.allclose(post.sum(-1), f.sum(-1), rtol=1e-14, atol=0)
    assert torch.allclose(post @ cmr.C, f @ cmr.C, rtol=0, atol=1e-15)
    feq = _feq_textbook(rho, u)
    post_eq, _, _ = cmr.collide(feq, S)
    assert torch.allclose(post_eq, feq, rtol=0, atol=1e-14)


def test_collision_relaxes_shear_stress_by_one_minus_s():
    """The off-diagonal second central moment relaxes towards 0 at rate S_4."""
    rho, u = _rand_state(64, 10)
    g = torch.Generator().manual_seed(11)
    f = _feq_textbook(rho, u) * (1 + 0.05 * (2 * torch.rand(64, 27, generator=g, dtype=DT) - 1))
    nu = 0.02
    S = cmr.relaxation_rates(nu)
    post, _, _ = cmr.collide(f, S)
    cb = cmr.C - u[:, None, :]
    rho_f = f.sum(-1)
    u_f = (f @ cmr.C) / rho_f[:, None]
    cb = cmr.C - u_f[:, None, :]
    pre_xy = (cb[..., 0] * cb[..., 1] * f).sum(-1)
    post_xy = (cb[..., 0] * cb[..., 1] * post).sum(-1)
    s = 1.0 / (3 * nu + 0.5)
    assert torch.allclose(post_xy, (1 - s) * pre_xy, rtol=0, atol=1e-16)


# ------------------------------------------------------------------ adaptive relaxation

def test_adaptive_factor_on_linear_and_quadratic_shear():
    n = 12
    y = torch.arange(n, dtype=DT)
    for s in (0.02, 0.08, 0.3):
        u = torch.zeros(3, n, n, n, dtype=DT)
        u[0] = s * y[None, :, None]                     # du_x/dy = s exactly
        zz, yy, xx = torch.meshgrid(torch.arange(1, n - 1), torch.arange(1, n - 1),
                                    torch.arange(1, n - 1), indexing="ij")
        g = grid.lagged_gradient_norm(u, (False,) * 3, zz.flatten(), yy.flatten(), xx.flatten())
        assert torch.allclose(g, torch.full_like(g, s), rtol=1e-14, atol=0)
        phi = cmr.adaptive_factor(g)
        expect = -4.0 * min(s / 0.1, 1.0) + 5.0
        assert torch.allclose(phi, torch.full_like(phi, expect), rtol=1e-14, atol=0)
    # quadratic field: central differences are exact, u_x = y^2 -> du_x/dy = 2y
    u = torch.zeros(3, n, n, n, dtype=DT)
    u[0] = 1e-3 * (y ** 2)[None, :, None]
    g = grid.lagged_gradient_norm(u, (False,) * 3, torch.tensor([5]), torch.tensor([4]),
                                  torch.tensor([6]))
    assert g.item() == pytest.approx(2e-3 * 4, rel=1e-13)


def test_local_strain_estimate_on_a_decaying_shear_wave():
    """The local estimate of |grad u| from non-equilibrium moments (Sec. 4.2.1 relation)
    reproduces |du_x/dy| = A k |cos(k y)| exp(-nu k^2 t) of a periodic shear wave once the
    start-up transient has decayed; a missing factor of S or rho would miss by > 20 %."""
    n = 32
    b = synth._empty_block((2, n, 2))
    A, k = 0.04, 2 * math.pi / n
    y = np.arange(n)
    b.u0[0] = (A * np.sin(k * y))[None, :, None]
    st = grid.init_state(b.rho0, b.u0, b.c0, b.flags)
    nu = 0.02
    p = grid.Params(nu=nu, periodic=(True, True, True), adaptive=False)
    t = 60
    st = grid.run(st, p, t)
    # the populations entering step t+1 at x = z = 0, all y
    zz = torch.zeros(n, dtype=torch.long)
    yy = torch.arange(n)
    nxt = {o: grid.neighbour_index(n, True, o) for o in (-1, 0, 1)}
    cols = []
    for q in range(27):
        cx, cy, cz = (int(v) for v in cmr.C[q])
        cols.append(st.f[q, 0, nxt[-cy][yy], 0])
    f_in = torch.stack(cols, dim=-1)
    g = grid.local_strain_norm(f_in, nu).numpy()
    exact = A * k * np.abs(np.cos(k * (y + 0.0))) * math.exp(-nu * k * k * (t + 0.5))
    big = exact > 0.5 * exact.max()
    assert np.allclose(g[big], exact[big], rtol=5e-3)


# ------------------------------------------------------------------------- flows

def _state(scene):
    b = scene.blocks[0]
    return grid.init_state(b.rho0, b.u0, b.c0, b.flags)


def test_uniform_flow_is_exact_on_periodic_and_open_boxes():
    for per in ((True, True, True), (False, False, False)):
        b = synth._empty_block((6, 5, 4))
        b.u0[0], b.u0[1], b.u0[2] = 0.07, -0.02, 0.03
        st = grid.init_state(b.rho0, b.u0, b.c0, b.flags)
        p = grid.Params(nu=0.01, periodic=per)
        f0 = st.f.clone()
        for _ in range(3):
            st = grid.step(st, p)
        assert torch.allclose(st.f, f0, rtol=0, atol=1e-15)


def test_periodic_run_conserves_mass_and_momentum():
    sc = synth.random_scene(dims=(8, 7, 6), seed=3, nu=0.01)
    st = _state(sc)
    p = grid.Params(nu=sc.nu, periodic=sc.periodic)
    r0 = grid.reductions(st)
    for _ in range(5):
        st = grid.step(st, p)
    r1 = grid.reductions(st)
    assert abs(r1[0] - r0[0]) / r0[0] < 1e-14
    assert torch.allclose(r1[1:4], r0[1:4], rtol=0, atol=1e-13)


def test_bounce_back_box_conserves_mass():
    sc = synth.random_scene(dims=(10, 9, 8), seed=4, nu=0.02,
                            spheres=[(4.0, 4.0, 4.0, 2.5)])
    b = sc.blocks[0]
    b.flags[:, :, 0] |= synth.SOLID       # closed walls on two faces; periodic elsewhere
    b.flags[:, :, -1] |= synth.SOLID
    st = _state(sc)
    p = grid.Params(nu=sc.nu, periodic=(True, True, True))
    m0 = grid.reductions(st)[0]
    for _ in range(6):
        st = grid.step(st, p)
    assert abs(grid.reductions(st)[0] - m0) / m0 < 1e-14


def test_plane_poiseuille_profile():
    """Body-force-driven channel between halfway bounce-back walls: the steady profile is
    u(y) = F/(2 nu) (y - y0)(y1 - y) with the walls at the half links y0, y1."""
    H = 16
    ny = H + 2
    nu = 1.0 / 6.0
    F = 1e-6
    flags = np.zeros((1, ny, 1), np.uint8)
    flags[0, 0, 0] = flags[0, ny - 1, 0] = synth.SOLID
    st = grid.init_state(np.ones((1, ny, 1)), np.zeros((3, 1, ny, 1)), np.zeros((1, ny, 1)), flags)
    p = grid.Params(nu=nu, periodic=(True, True, True), body_force=(F, 0.0, 0.0))
    st = grid.run(st, p, 1100)
    rho, u = grid.macros_field(st)
    u_phys = u[0, 0, 1:-1, 0] + F / (2 * rho[0, 1:-1, 0])
    yv = torch.arange(1, H + 1, dtype=DT)
    ua = F / (2 * nu) * (yv - 0.5) * (H + 0.5 - yv)
    assert (torch.linalg.norm(u_phys - ua) / torch.linalg.norm(ua)).item() < 0.01


def test_taylor_green_decay_rate_matches_viscosity():
    """z-invariant Taylor-Green vortex: after the start-up transient of the equilibrium
    initialisation, the mode amplitude decays as exp(-2 nu k^2 t) and the kinetic energy
    as exp(-4 nu k^2 t).  (nz = 2 is exact for a z-invariant periodic flow.)"""
    n = 32
    sc = synth.taylor_green(n, nz=2)
    st = _state(sc)
    p = grid.Params(nu=sc.nu, periodic=sc.periodic)
    k = 2 * math.pi / n
    x = torch.arange(n, dtype=DT)
    basis = (torch.sin(k * x)[None, None, :] * torch.cos(k * x)[None, :, None]).expand(2, n, n)

    def amp(s):
        _, u = grid.macros_field(s)
        return (u[0] * basis).sum().item() / (basis * basis).sum().item()

    E0 = grid.reductions(st)[4].item()
    log = {}
    for t in range(1, 201):
        st = grid.step(st, p)
        if t in (60, 200):
            log[t] = (amp(st), grid.reductions(st)[4].item())
    rate = -math.log(log[200][0] / log[60][0]) / 140.0
    assert rate == pytest.approx(2 * sc.nu * k * k, rel=5e-3)
    e_ratio = log[200][1] / log[60][1]
    assert e_ratio == pytest.approx(math.exp(-4 * sc.nu * k * k * 140), rel=5e-3)
    # whole-run energy against the closed form, start-up loss included
    assert log[200][1] / E0 == pytest.approx(math.exp(-4 * sc.nu * k * k * 200), rel=0.03)


# --------------------------------------------------------------------- node kinds

def test_inflow_and_solid_nodes_hold_their_equilibria():
    sc = synth.random_scene(dims=(8, 8, 8), seed=5, periodic=(False, False, False),
                            spheres=[(5.0, 4.0, 4.0, 1.6)], inflow=(4, 4, 2.5, 0.1))
    st = _state(sc)
    p = grid.Params(nu=0.01, periodic=sc.periodic)
    st1 = grid.step(st, p)
    fl = st.flags
    inflow = (fl & synth.INFLOW) != 0
    solid = (fl & synth.SOLID) != 0
    assert inflow.any() and solid.any()
    u_in = sc.blocks[0].u0[:, inflow.numpy()].T
    feq = _feq_textbook(torch.ones(u_in.shape[0], dtype=DT), torch.as_tensor(u_in))
    assert torch.allclose(st1.f[:, inflow].T, feq, atol=1e-15, rtol=0)
    w = _weights()
    assert torch.allclose(st1.f[:, solid].T, w.expand(int(solid.sum()), 27), atol=1e-15, rtol=0)
    assert (st1.u[:, solid] == 0).all()
    assert (st1.c[(fl & synth.SCALAR_SRC) != 0] == 1.0).all()


# ------------------------------------------------------------------------ scalar

def test_scalar_advection_linear_profile_is_exact():
    """A linear scalar profile advected by a uniform flow shifts by exactly u per step
    (trilinear interpolation is exact on affine data)."""
    b = synth._empty_block((12, 6, 5))
    ux = 0.3
    b.u0[0] = ux
    xs = np.arange(12)[None, None, :]
    b.c0[:] = np.broadcast_to(0.5 + 0.1 * xs, b.c0.shape)
    st = grid.init_state(b.rho0, b.u0, b.c0, b.flags)
    p = grid.Params(nu=0.05, periodic=(False, True, True))
    st1 = grid.step(st, p)
    interior = st1.c[:, :, 1:]
    expect = torch.as_tensor(0.5 + 0.1 * (np.arange(1, 12) - ux))[None, None, :].expand_as(interior)
    assert torch.allclose(interior, expect, rtol=0, atol=1e-14)
    assert torch.allclose(st1.c[:, :, 0], torch.full_like(st1.c[:, :, 0], 0.5), atol=1e-15)


def test_trilinear_sampling_is_exact_on_affine_fields_and_wraps():
    g = torch.Generator().manual_seed(12)
    Z, Y, X = 5, 6, 7
    zz, yy, xx = torch.meshgrid(torch.arange(Z, dtype=DT), torch.arange(Y, dtype=DT),
                                torch.arange(X, dtype=DT), indexing="ij")
    c = 0.3 + 0.02 * xx - 0.05 * yy + 0.07 * zz
    px = 0.5 + 5.0 * torch.rand(50, generator=g, dtype=DT)
    py = 0.5 + 4.0 * torch.rand(50, generator=g, dtype=DT)
    pz = 0.5 + 3.0 * torch.rand(50, generator=g, dtype=DT)
    got = grid.sample_trilinear(c, px, py, pz, (False, False, False))
    assert torch.allclose(got, 0.3 + 0.02 * px - 0.05 * py + 0.07 * pz, atol=1e-15, rtol=0)
    # periodic wrap: sampling at x = -0.25 mixes the last and first columns
    got = grid.sample_trilinear(c, torch.tensor([-0.25], dtype=DT), torch.tensor([2.0], dtype=DT),
                                torch.tensor([1.0], dtype=DT), (True, True, True))
    want = 0.25 * c[1, 2, X - 1] + 0.75 * c[1, 2, 0]
    assert got.item() == pytest.approx(want.item(), abs=1e-15)
