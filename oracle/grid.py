"""FP64 reference for one uniform block: pull-stream, boundaries, CMR collision with the
adaptive high-order relaxation, and passive-scalar advection.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Per step and per node x (LBE of Sec. 1 / Appendix, iterated in pull form):
  1. f_i^in(x) = f~_i(x - c_i); if x - c_i is an obstacle voxel the population is
     reflected, f_i^in(x) = f~_opp(i)(x) (halfway bounce-back with the wall at rest; the
     paper names bounce-back as the first-order wall treatment in Sec. 6.1).  Outside the
     block, a periodic axis wraps and an open axis clamps the source node into the block
     (zero-gradient / Neumann copy, Sec. 6.1 uses Neumann for open boundaries).
  2. rho, u from f^in (Sec. 1).
  3. adaptive factor (Sec. 4.1) from |grad u|, the Frobenius norm of the central-difference
     Jacobian of the velocity field stored by the previous step (neighbour indices wrap or
     clamp as in 1; obstacle voxels store u = 0).
  4. f~ = f^in - T S (m - m^eq)  (Sec. 3.1, dense solve in ``oracle.cmr``).
  1b. No-slip walls (Sec. 6.1's second-order wall, read as the regularized on-node wall):
     on wall faces of the block, and, with ``obstacle_walls``, on the surface voxels of the
     obstacles (obstacle voxels with a non-obstacle pull source), which then are active wall
     nodes at rest while only the inner voxels stay inert; see ``regularized_wall``.
  5. Obstacle voxels hold the rest equilibrium and u = 0; inflow nodes hold the
     equilibrium T m^eq(1, u_in) (Dirichlet inflow of Sec. 6.1) with u_in their stored
     velocity; ghost nodes of refined blocks are left untouched (they belong to the
     coarse-to-fine mapping).
  6. Passive scalar (stands in for the paper's smoke particles, Sec. 6.4): semi-Lagrangian
     c^{n+1}(x) = trilinear sample of c^n at x - u^{n+1}(x) (periodic wrap or clamp to the
     block; each displacement component limited to one node, which only matters for the
     non-physical |u| >= 1); source nodes are reset to c_src; obstacle voxels hold 0.

An optional ``body_force`` (test-only; not part of the paper's solver) adds the
exact-difference forcing f += f^eq(rho, u + F/rho) - f^eq(rho, u) after the collision; it
exists only to pin the plane-Poiseuille closed form.
"""
from __future__ import annotations

import dataclasses
from typing import Optional, Sequence

import numpy as np
import torch

from . import cmr
from .cmr import C, DT, OPP

SOLID, INFLOW, SCALAR_SRC, GHOST = 1, 2, 4, 8


@dataclasses.dataclass
class Params:
    nu: float
    periodic: Sequence[bool] = (True, True, True)
    adaptive: bool = True
    a: float = cmr.A_DEFAULT
    b: float = cmr.B_DEFAULT
    g_max: float = cmr.G_MAX_DEFAULT
    nu_hi: Sequence[float] = cmr.NU_HI_DEFAULT
    c_src: float = 1.0
    body_force: Optional[Sequence[float]] = None
    grad_mode: str = "lagged"    # "lagged" central differences of the stored velocity, or
                                 # "local" strain rate from the node's non-equilibrium moments
    walls: Sequence[bool] = (False,) * 6   # no-slip wall faces x-, x+, y-, y+, z-, z+
    obstacle_walls: bool = False   # obstacle surfaces as regularized on-node walls


@dataclasses.dataclass
class State:
    f: torch.Tensor       # (27, Z, Y, X) post-collision populations f~
    u: torch.Tensor       # (3, Z, Y, X) velocity stored by the last step
    c: torch.Tensor       # (Z, Y, X) passive scalar
    flags: torch.Tensor   # (Z, Y, X) uint8

    def clone(self):
        return State(self.f.clone(), self.u.clone(), self.c.clone(), self.flags.clone())


def neighbour_index(n: int, periodic: bool, offset: int) -> torch.Tensor:
    """Index of node k + offset along one axis: wrapped (periodic) or clamped (open)."""
    k = torch.arange(n) + offset
    return torch.remainder(k, n) if periodic else torch.clamp(k, 0, n - 1)


def init_state(rho0, u0, c0, flags) -> State:
    """f_0 = T m^eq(rho_0, u_0) on every node (Algorithm 1, Sec. 6.1); obstacle voxels get
    the rest state with u = 0."""
    def as_t(a):
        return a.to(DT) if isinstance(a, torch.Tensor) else torch.as_tensor(np.asarray(a), dtype=DT)

    rho0, u0, c0 = as_t(rho0), as_t(u0), as_t(c0)
    flags = torch.as_tensor(np.asarray(flags).astype(np.uint8)) \
        if not isinstance(flags, torch.Tensor) else flags
    solid = (flags & SOLID) != 0
    rho = torch.where(solid, torch.ones_like(rho0), rho0)
    u0 = torch.where(solid[None], torch.zeros_like(u0), u0)
    c0 = torch.where(solid, torch.zeros_like(c0), c0)
    f = cmr.equilibrium(rho.reshape(-1), u0.reshape(3, -1).T).T.reshape((27,) + rho.shape)
    return State(f.contiguous(), u0, c0, flags)


def sample_trilinear(c: torch.Tensor, px, py, pz, periodic) -> torch.Tensor:
    """Trilinear interpolation of c[z][y][x] at node-unit positions (px, py, pz)."""
    Z, Y, X = c.shape
    idx, wts = [], []
    for p, n, per in ((px, X, periodic[0]), (py, Y, periodic[1]), (pz, Z, periodic[2])):
        if per:
            fl = torch.floor(p)
            t = p - fl
            i0 = torch.remainder(fl.long(), n)
            i1 = torch.remainder(i0 + 1, n)
        else:
            p = torch.clamp(p, 0.0, float(n - 1))
            if n > 1:
                i0 = torch.clamp(torch.floor(p).long(), max=n - 2)
            else:
                i0 = torch.zeros_like(p, dtype=torch.long)
            t = p - i0.to(DT)
            i1 = torch.clamp(i0 + 1, max=n - 1)
        idx.append((i0, i1))
        wts.append((1.0 - t, t))
    out = torch.zeros_like(px)
    for bz in (0, 1):
        for by in (0, 1):
            for bx in (0, 1):
                w = wts[0][bx] * wts[1][by] * wts[2][bz]
                out = out + w * c[idx[2][bz], idx[1][by], idx[0][bx]]
    return out


def face_unknowns(walls, dims, x, y, z) -> torch.Tensor:
    """(K, 27) mask of the populations of the listed nodes whose pull source lies beyond a
    wall face of the block."""
    n = dims
    coord = (x, y, z)
    unk = torch.zeros((x.shape[0], 27), dtype=torch.bool)
    for q in range(27):
        col = torch.zeros(x.shape, dtype=torch.bool)
        for a in range(3):
            ca = int(C[q, a])
            if walls[2 * a] and ca == 1:
                col |= coord[a] == 0
            if walls[2 * a + 1] and ca == -1:
                col |= coord[a] == n[a] - 1
        unk[:, q] = col
    return unk


def surface_voxels(flags: torch.Tensor, periodic) -> torch.Tensor:
    """Obstacle voxels with at least one non-obstacle node among their pull sources (the 26
    neighbours, wrapped on periodic axes and clamped on open ones)."""
    Z, Y, X = flags.shape
    solid = (flags & SOLID) != 0
    nx = {o: neighbour_index(X, periodic[0], o) for o in (-1, 0, 1)}
    ny = {o: neighbour_index(Y, periodic[1], o) for o in (-1, 0, 1)}
    nz = {o: neighbour_index(Z, periodic[2], o) for o in (-1, 0, 1)}
    open_nb = torch.zeros_like(solid)
    for q in range(27):
        cx, cy, cz = (int(v) for v in C[q])
        open_nb |= ~solid[nz[-cz]][:, ny[-cy]][:, :, nx[-cx]]
    return solid & open_nb


def regularized_wall(f_in: torch.Tensor, unk: torch.Tensor, node=None) -> torch.Tensor:
    """Second-order no-slip wall (Sec. 6.1, read as the regularized on-node wall of the
    cited method), applied to the pulled populations f_in (K, 27) of the listed nodes; unk
    (K, 27) marks the populations whose pull source lies beyond the wall (outside a wall face
    of the block, or inside an obstacle whose surface voxels are the wall nodes).  An unknown
    population is completed by bounce-back from its opposite (the wall is at rest); where the
    opposite is unknown too (edges, corners) both take the rest equilibrium w_i rho.  rho is
    the mass of the completed set (for one wall: sum_{c.n = 0} f + 2 sum_{c.n < 0} f).  All
    27 populations of a wall node (``node`` (K,), by default the nodes with an unknown
    population; a surface voxel is a wall node even when nothing reaches it from inside the
    obstacle) are then rebuilt from the equilibrium at (rho, u = 0) and the non-equilibrium
    stress Pi of the completed set, f_i = w_i rho + w_i / (2 c_s^4) Q_i : Pi with
    Q_i = c_i c_i - c_s^2 I."""
    if node is None:
        node = unk.any(dim=1)
    if not bool(node.any()):
        return f_in
    W = cmr.equilibrium(torch.ones(1, dtype=DT), torch.zeros(1, 3, dtype=DT))[0]   # weights
    unk_opp = unk[:, OPP]
    both = unk & unk_opp
    f_c = torch.where(unk & ~unk_opp, f_in[:, OPP], f_in)
    rho = torch.where(both, torch.zeros_like(f_c), f_c).sum(1) / (1.0 - (W * both).sum(1))
    feq = W[None, :] * rho[:, None]
    f_c = torch.where(both, feq, f_c)
    pi = torch.einsum("kq,qa,qb->kab", f_c - feq, C, C)
    Q = C[:, :, None] * C[:, None, :] - torch.eye(3, dtype=DT)[None] / 3.0
    f_reg = feq + 4.5 * W[None, :] * torch.einsum("qab,kab->kq", Q, pi)
    return torch.where(node[:, None], f_reg, f_in)


def lagged_gradient_norm(u: torch.Tensor, periodic, z, y, x) -> torch.Tensor:
    """|grad u| at the listed nodes: Frobenius norm of the central-difference Jacobian
    d u_a / d x_b ~ (u_a(x + e_b) - u_a(x - e_b)) / 2 of a stored velocity field, with
    neighbour indices wrapped (periodic) or clamped (open) as in the pull."""
    _, Z, Y, X = u.shape
    nx = {o: neighbour_index(X, periodic[0], o) for o in (-1, 1)}
    ny = {o: neighbour_index(Y, periodic[1], o) for o in (-1, 1)}
    nz = {o: neighbour_index(Z, periodic[2], o) for o in (-1, 1)}
    g2 = torch.zeros(z.shape, dtype=DT)
    for a in range(3):
        g2 = g2 + (0.5 * (u[a, z, y, nx[1][x]] - u[a, z, y, nx[-1][x]])) ** 2
        g2 = g2 + (0.5 * (u[a, z, ny[1][y], x] - u[a, z, ny[-1][y], x])) ** 2
        g2 = g2 + (0.5 * (u[a, nz[1][z], y, x] - u[a, nz[-1][z], y, x])) ** 2
    # the floor only keeps reverse-mode differentiation finite where the gradient is exactly
    # zero (the value changes by less than 1e-149)
    return torch.sqrt(torch.clamp(g2, min=1e-300))


def local_strain_norm(f_in: torch.Tensor, nu: float) -> torch.Tensor:
    """|grad u| estimated from a node's own pre-collision populations: the non-equilibrium
    second central moments Pi = m - m^eq (moments 4..9 of the Appendix basis) give the strain
    rate through Pi^(1) = -2 c_s^2 rho S_hat / S (Sec. 4.2.1, with S the shear rate of
    Sec. 3.1 Eq. 3 and c_s^2 = 1/3); the norm is sqrt(2 S_hat : S_hat), which equals |grad u|
    for a shear flow."""
    rho, u = cmr.macros(f_in)
    m = (cmr.moment_matrix(u).transpose(-1, -2) @ f_in[..., None])[..., 0]
    mn = m - cmr.m_eq(rho, u)
    pxy, pxz, pyz = mn[..., 4], mn[..., 5], mn[..., 6]
    pxx = (mn[..., 9] + mn[..., 7] + mn[..., 8]) / 3.0
    pyy = (mn[..., 9] - 2.0 * mn[..., 7] + mn[..., 8]) / 3.0
    pzz = (mn[..., 9] + mn[..., 7] - 2.0 * mn[..., 8]) / 3.0
    S = 1.0 / (3.0 * nu + 0.5)
    scale = -3.0 * S / (2.0 * rho)
    ss = (pxx ** 2 + pyy ** 2 + pzz ** 2) + 2.0 * (pxy ** 2 + pxz ** 2 + pyz ** 2)
    return torch.sqrt(torch.clamp(2.0 * ss * scale * scale, min=1e-300))


def _forced_shift(rho, u, F):
    """Exact-difference forcing increment (test-only hook, see module docstring)."""
    Fv = torch.as_tensor(F, dtype=DT)
    return cmr.equilibrium(rho, u + Fv / rho[..., None]) - cmr.equilibrium(rho, u)


def step_cells(st: State, p: Params, z: torch.Tensor, y: torch.Tensor, x: torch.Tensor):
    """One step evaluated at the listed nodes only; returns (f~ (K,27), u (K,3), c (K,))."""
    Z, Y, X = st.c.shape
    per = p.periodic
    nx = {o: neighbour_index(X, per[0], o) for o in (-1, 0, 1)}
    ny = {o: neighbour_index(Y, per[1], o) for o in (-1, 0, 1)}
    nz = {o: neighbour_index(Z, per[2], o) for o in (-1, 0, 1)}
    solid = (st.flags & SOLID) != 0
    surface = torch.zeros_like(solid)
    if p.obstacle_walls:          # surface voxels are wall nodes; only the interior is inert
        surface = surface_voxels(st.flags, per)
        solid = solid & ~surface
    fl = st.flags[z, y, x]
    wall_node = surface[z, y, x]

    # 1. pull with halfway bounce-back (from inert obstacle voxels)
    cols, from_solid = [], []
    for q in range(27):
        cx, cy, cz = (int(v) for v in C[q])
        sz, sy, sx = nz[-cz][z], ny[-cy][y], nx[-cx][x]
        from_wall = solid[sz, sy, sx]
        from_solid.append(from_wall)
        cols.append(torch.where(from_wall, st.f[OPP[q], z, y, x], st.f[q, sz, sy, sx]))
    f_in = torch.stack(cols, dim=-1)
    if any(p.walls) or p.obstacle_walls:
        unk = face_unknowns(p.walls, (X, Y, Z), x, y, z)
        node = unk.any(dim=1) | wall_node
        unk |= torch.stack(from_solid, dim=-1) & wall_node[:, None]
        f_in = regularized_wall(f_in, unk, node)

    # 3. adaptive factor from the lagged velocity field
    if p.adaptive and p.grad_mode == "local":
        phi = cmr.adaptive_factor(local_strain_norm(f_in, p.nu), p.a, p.b, p.g_max)
    elif p.adaptive:
        phi = cmr.adaptive_factor(lagged_gradient_norm(st.u, per, z, y, x), p.a, p.b, p.g_max)
    else:
        phi = torch.ones(z.shape, dtype=DT)
    S = cmr.relaxation_rates(p.nu, phi, p.nu_hi)

    # 2 + 4. macros and CMR collision
    f_post, rho, u = cmr.collide(f_in, S)
    if p.body_force is not None:
        f_post = f_post + _forced_shift(rho, u, p.body_force)

    # 5. node kinds (selected with where, so the step stays differentiable)
    is_solid = ((fl & SOLID) != 0) & ~wall_node
    is_in = ((fl & INFLOW) != 0) & ~is_solid
    is_ghost = (fl & GHOST) != 0
    u_own = st.u[:, z, y, x].T
    if bool(is_in.any()):
        f_in_eq = cmr.equilibrium(torch.ones(z.shape, dtype=DT), u_own)
        f_post = torch.where(is_in[:, None], f_in_eq, f_post)
        u = torch.where(is_in[:, None], u_own, u)
    if bool(is_solid.any()):
        f_rest = cmr.equilibrium(torch.ones(1, dtype=DT), torch.zeros(1, 3, dtype=DT))
        f_post = torch.where(is_solid[:, None], f_rest, f_post)
        u = torch.where(is_solid[:, None], torch.zeros_like(u), u)
    if bool(is_ghost.any()):
        f_post = torch.where(is_ghost[:, None], st.f[:, z, y, x].T, f_post)
        u = torch.where(is_ghost[:, None], u_own, u)

    # 6. passive scalar (departure point at most one node away: |u| < 1 in any stable run)
    dsp = torch.clamp(-u, -1.0, 1.0)
    c_new = sample_trilinear(st.c, x.to(DT) + dsp[:, 0], y.to(DT) + dsp[:, 1],
                             z.to(DT) + dsp[:, 2], per)
    c_new = torch.where((fl & SCALAR_SRC) != 0, torch.full_like(c_new, p.c_src), c_new)
    c_new = torch.where(is_solid, torch.zeros_like(c_new), c_new)
    c_new = torch.where(is_ghost, st.c[z, y, x], c_new)
    return f_post, u, c_new


def step(st: State, p: Params, chunk: int = 1 << 15) -> State:
    """Advance the whole block by one step (all nodes, evaluated in chunks)."""
    Z, Y, X = st.c.shape
    zz, yy, xx = torch.meshgrid(torch.arange(Z), torch.arange(Y), torch.arange(X), indexing="ij")
    zz, yy, xx = zz.reshape(-1), yy.reshape(-1), xx.reshape(-1)
    fs, us, cs = [], [], []
    for s in range(0, zz.numel(), chunk):
        e = min(s + chunk, zz.numel())
        fo, uo, co = step_cells(st, p, zz[s:e], yy[s:e], xx[s:e])
        fs.append(fo)
        us.append(uo)
        cs.append(co)
    f_out, u_out, c_out = torch.cat(fs), torch.cat(us), torch.cat(cs)
    return State(f_out.T.reshape(27, Z, Y, X).contiguous(), u_out.T.reshape(3, Z, Y, X).contiguous(),
                 c_out.reshape(Z, Y, X), st.flags)


def run(st: State, p: Params, steps: int, callback=None) -> State:
    for n in range(steps):
        st = step(st, p)
        if callback is not None:
            callback(n + 1, st)
    return st


def macros_field(st: State):
    """(rho, u) of the stored post-collision state, per node."""
    rho = st.f.sum(0)
    u = torch.einsum("qzyx,qa->azyx", st.f, C) / rho
    return rho, u


def reductions(st: State):
    """FP64 diagnostics over fluid + inflow nodes: mass, momentum (3), kinetic energy."""
    rho, u = macros_field(st)
    keep = ((st.flags & (SOLID | GHOST)) == 0).to(DT)
    mass = (rho * keep).sum()
    mom = (rho * u * keep).sum(dim=(1, 2, 3))
    ke = 0.5 * (rho * (u * u).sum(0) * keep).sum()
    return torch.stack([mass, mom[0], mom[1], mom[2], ke])
