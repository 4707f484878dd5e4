"""FP64 reference of the continuous-scale coupling (Sec. 3.2, Sec. 4.2, Algorithm 1).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Blocks.  Block 0 is the reference scale s0 (h = 1, node k at k).  Every other block b is a
uniform grid of spacing h_b < 1 (in reference units) whose node k sits at o_b + k h_b; its
outermost node layer is the scale boundary (ghost layer), written only by prior-mapping.
Per block: nu_b = nu_0 / h_b, from the Reynolds-number invariance
1/S^f - 1/2 = alpha (1/S^c - 1/2) (Sec. 3.2, Eq. 4); the high-order rates use the same nu'
table in every block's own lattice units; velocity and density are the same numbers on
every scale because dt_s = dx_s (Sec. 4.2.4).

Mapping between scales (Sec. 3.2, Eq. 9-11; Sec. 4.2.1): for post-collision f of scale s_i
moved to scale s_j,
    f^{s_j} = T (m^eq + K_hat (m - m^eq)),  m = M(u)^T f,  m^eq = m^eq(rho, u),
    K_hat = (I - S^{s_j}) K (I - S^{s_i})^{-1},  diag K = S^{s_i}_k / (alpha S^{s_j}_k) for
    k = 4..8 and 1 otherwise,  alpha = dx_{s_i} / dx_{s_j}.
With the per-block high-order rates equal on both sides, K_hat_k = 1 for k outside 4..8.

Readings (the paper is silent or ambiguous):
  * Spatial interpolation is trilinear over the 8 nodes of the source cell containing the
    point (Sec. 4.2.2); corners that are obstacle voxels of the source are dropped and the
    remaining weights renormalised; if all 8 are obstacles, a scale-boundary (ghost) node
    takes the rest state (rho = 1, u = 0, scalar 0: it has no dynamics of its own to keep)
    and a post-mapped node is left unchanged (it keeps its own update).
  * Prior-mapping source: the nearest coarser block that contains the whole target block
    (Sec. 4.2.5 chooses the nearest coarser scale per node; for nested blocks this is the
    same block).  Post-mapping targets: every coarser block (Sec. 4.2.5), at its nodes that
    lie in the target's interior span [o + h, o + (N-2) h] on every axis, that are neither
    its own ghost nodes nor obstacle voxels.
  * Sub-steps l = ceil(1/h - 1e-9): for a non-integer ratio this equals floor(1/h) + 1 of
    Sec. 4.2.4; for an integer ratio it lands exactly on t_n + dt_0 and no temporal
    interpolation is needed.
  * Before sub-step j (j = 1..l) the ghost layer holds the mapping of the source scale at
    time t_n + (j-1) h, linearly interpolated between the source's states at t_n and
    t_n + dt_0 (Sec. 4.2.4); a pull step reads the ghost layer at the start of the sub-step.
    The j = 1 mapping refreshes the ghost layer of the block's t_n state (its source may
    have been post-mapped since), and that refreshed state is the t_n source of finer
    blocks.
  * Temporal alignment (Sec. 4.2.4): the block's interior at t_n + dt_0 is the quadratic
    Lagrange interpolant through its states at t_n, t_n + (l-1) h and t_n + l h; the
    stored velocity is recomputed from the interpolated populations and the scalar is
    interpolated alike; the ghost layer is the mapping of the source at t_n + dt_0.  The
    block's clock is then aligned with s0.  Every node the sub-steps update is aligned,
    the obstacles' surface voxels too when they are walls (they are updated wall nodes);
    inert obstacle voxels and ghost nodes keep their last state.
  * Ghost and post-mapped nodes carry the velocity of their mapped populations (the
    mapping keeps rho and u) and the trilinearly interpolated scalar.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List

import numpy as np
import torch

from . import cmr, grid
from .cmr import DT

SOLID, INFLOW, SCALAR_SRC, GHOST = grid.SOLID, grid.INFLOW, grid.SCALAR_SRC, grid.GHOST


@dataclasses.dataclass
class Blk:
    origin: np.ndarray      # (3,) reference units, (x, y, z)
    h: float
    dims: tuple             # (nx, ny, nz)
    state: grid.State
    params: grid.Params
    substeps: int = 1
    integer_ratio: bool = True
    parent: int = -1
    far: bool = False       # far-field block (h > 1) around `child`
    child: int = -1

    def interior_lo_hi(self):
        lo = self.origin + self.h
        hi = self.origin + (np.array(self.dims) - 2) * self.h
        return lo, hi


def put_nodes(st: grid.State, z, y, x, f_rows, u_rows, c_vals) -> grid.State:
    """A copy of st with the listed nodes' populations (K, 27), velocities (K, 3) and
    scalars (K,) replaced (out of place, so reverse-mode differentiation can run through)."""
    _, Z, Y, X = st.f.shape
    lin = (z * Y + y) * X + x
    f = st.f.reshape(27, -1).index_copy(1, lin, f_rows.T.to(st.f.dtype)).reshape(st.f.shape)
    u = st.u.reshape(3, -1).index_copy(1, lin, u_rows.T.to(st.u.dtype)).reshape(st.u.shape)
    c = st.c.reshape(-1).index_copy(0, lin, c_vals.to(st.c.dtype)).reshape(st.c.shape)
    return grid.State(f, u, c, st.flags)


def rest_nodes(st: grid.State, z, y, x) -> grid.State:
    """Scale-boundary nodes whose source corners are all obstacle voxels: no value can be
    interpolated, so they take the rest state (rho = 1, u = 0, scalar 0)."""
    if z.numel() == 0:
        return st
    feq = cmr.equilibrium(torch.ones(1, dtype=DT), torch.zeros(1, 3, dtype=DT))
    k = z.numel()
    return put_nodes(st, z, y, x, feq.expand(k, 27), torch.zeros(k, 3, dtype=DT),
                     torch.zeros(k, dtype=DT))


def shear_rate(nu: float) -> float:
    return 1.0 / (3.0 * nu + 0.5)


def k_hat(src: Blk, dst: Blk) -> torch.Tensor:
    """Diagonal of K_hat^{src -> dst} (Sec. 3.2)."""
    Ss, Sd = shear_rate(src.params.nu), shear_rate(dst.params.nu)
    alpha = src.h / dst.h
    if abs(1.0 - Ss) < 1e-12 or abs(1.0 - Sd) < 1e-12:
        raise ValueError("K_hat undefined for S = 1 (nu = 1/6)")
    K = torch.ones(27, dtype=DT)
    K[4:9] = (1.0 - Sd) * (Ss / (alpha * Sd)) / (1.0 - Ss)
    return K


def map_populations(f: torch.Tensor, K: torch.Tensor) -> torch.Tensor:
    """f' = T (m^eq + K_hat (m - m^eq)) with M, T evaluated at the velocity of f."""
    rho, u = cmr.macros(f)
    MT = cmr.moment_matrix(u).transpose(-1, -2)
    m = (MT @ f[..., None])[..., 0]
    meq = cmr.m_eq(rho, u)
    return torch.linalg.solve(MT, (meq + K * (m - meq))[..., None])[..., 0]


def node_positions(b: Blk, z, y, x) -> torch.Tensor:
    """Reference-unit positions (K, 3) of the listed nodes of block b."""
    o = torch.as_tensor(b.origin, dtype=DT)
    return torch.stack([o[0] + b.h * x.to(DT), o[1] + b.h * y.to(DT), o[2] + b.h * z.to(DT)], -1)


def interpolate(src: Blk, f_src: torch.Tensor, c_src: torch.Tensor, pos: torch.Tensor):
    """Trilinear interpolation of populations (27,Z,Y,X) and scalar (Z,Y,X) of block src at
    reference-unit points pos (K,3), dropping obstacle corners.  Returns (f (K,27), c (K,),
    ok (K,) bool)."""
    nx, ny, nz = src.dims
    q = (pos - torch.as_tensor(src.origin, dtype=DT)) / src.h
    idx, wts = [], []
    for a, n in enumerate((nx, ny, nz)):
        i0 = torch.clamp(torch.floor(q[:, a]).long(), 0, max(n - 2, 0))
        t = q[:, a] - i0.to(DT)
        idx.append((i0, torch.clamp(i0 + 1, max=n - 1)))
        wts.append((1.0 - t, t))
    solid = (src.state.flags & SOLID) != 0
    f = torch.zeros(pos.shape[0], 27, dtype=DT)
    c = torch.zeros(pos.shape[0], dtype=DT)
    wsum = torch.zeros(pos.shape[0], dtype=DT)
    for bz in (0, 1):
        for by in (0, 1):
            for bx in (0, 1):
                zi, yi, xi = idx[2][bz], idx[1][by], idx[0][bx]
                w = wts[0][bx] * wts[1][by] * wts[2][bz]
                w = torch.where(solid[zi, yi, xi], torch.zeros_like(w), w)
                f = f + w[:, None] * f_src[:, zi, yi, xi].T
                c = c + w * c_src[zi, yi, xi]
                wsum = wsum + w
    ok = wsum > 0
    safe = torch.where(ok, wsum, torch.ones_like(wsum))
    return f / safe[:, None], c / safe, ok


class MultiScale:
    """A domain of blocks advanced by Algorithm 1."""

    def __init__(self, blocks: List[Blk]):
        self.blocks = blocks
        self.step_count = 0

    @staticmethod
    def build(scene, f32_inputs=True, obstacle_walls=False) -> "MultiScale":
        """Blocks of a ``synth.Scene``: block 0 is s0; refined blocks get ghost flags,
        nu_b = nu_0 / h_b, substep counts and their prior-mapping parent.  With
        ``obstacle_walls`` every block takes its obstacles' surface voxels as the
        second-order wall (``grid.Params.obstacle_walls``); the mappings keep treating every
        obstacle voxel as an obstacle (dropped corner, destination left alone)."""
        blocks = []
        for i, sb in enumerate(scene.blocks):
            conv = (lambda a: np.asarray(a, np.float32).astype(np.float64)) if f32_inputs \
                else (lambda a: np.asarray(a, np.float64))
            flags = sb.flags.copy()
            if i > 0:
                flags[0, :, :] |= GHOST
                flags[-1, :, :] |= GHOST
                flags[:, 0, :] |= GHOST
                flags[:, -1, :] |= GHOST
                flags[:, :, 0] |= GHOST
                flags[:, :, -1] |= GHOST
            st = grid.init_state(conv(sb.rho0), conv(sb.u0), conv(sb.c0), flags)
            h = float(sb.h)
            nu_b = scene.nu / h
            per = tuple(scene.periodic) if i == 0 else (False, False, False)
            p = grid.Params(nu=nu_b, periodic=per, adaptive=scene.adaptive, c_src=scene.c_src,
                            obstacle_walls=obstacle_walls)
            ratio = 1.0 / h
            l = max(1, math.ceil(ratio - 1e-9))
            blocks.append(Blk(origin=np.array(sb.origin, dtype=np.float64), h=h,
                              dims=tuple(sb.dims), state=st, params=p, substeps=l,
                              integer_ratio=abs(ratio - round(ratio)) < 1e-9))
        ms = MultiScale(blocks)
        for i in range(1, len(blocks)):
            blocks[i].parent = ms._containing_parent(i)
        return ms

    # ------------------------------------------------------------------ far field
    def outermost(self) -> int:
        """The block a new far-field block has to surround: the last far block, else s0."""
        far = [i for i, b in enumerate(self.blocks) if b.far]
        return far[-1] if far else 0

    @staticmethod
    def _outer_layer(dims):
        nx, ny, nz = dims
        m = torch.zeros((nz, ny, nx), dtype=torch.bool)
        m[0], m[-1], m[:, 0], m[:, -1], m[:, :, 0], m[:, :, -1] = (True,) * 6
        return m

    def set_outer_ghost(self, i: int, on: bool):
        """The outer layer of block i becomes (on) or stops being (off) a scale boundary,
        except its obstacle and inflow nodes, which keep their own update."""
        b = self.blocks[i]
        outer = self._outer_layer(b.dims)
        fl = b.state.flags
        keep = (fl & (SOLID | INFLOW)) != 0
        ghost = outer & ~keep if on else torch.zeros_like(outer)
        b.state.flags = torch.where(outer, torch.where(ghost, fl | GHOST, fl & ~GHOST), fl)

    def add_far_block(self, origin, h, dims, rho0, u0, c0, flags) -> int:
        """Far-field block (Sec. 4.2.4, 4.2.5): spacing h > 1, surrounding the outermost
        block, which from now on takes its outer layer from this block."""
        if not h > 1.0:
            raise ValueError("far-field blocks have h > 1")
        child = self.outermost()
        c = self.blocks[child]
        lo_c, hi_c = c.origin, c.origin + (np.array(c.dims) - 1) * c.h
        lo, hi = np.asarray(origin, float), np.asarray(origin, float) + (np.array(dims) - 1) * h
        if not (np.all(lo <= lo_c + 1e-9) and np.all(hi_c <= hi + 1e-9)):
            raise ValueError("a far-field block must contain the outermost block")
        ref = self.blocks[0].params
        p = grid.Params(nu=ref.nu / h, periodic=(False, False, False), adaptive=ref.adaptive,
                        c_src=ref.c_src, grad_mode=ref.grad_mode)
        conv = lambda a: np.asarray(a, np.float32).astype(np.float64)
        st = grid.init_state(conv(rho0), conv(u0), conv(c0), flags)
        self.blocks.append(Blk(origin=np.array(origin, dtype=np.float64), h=float(h),
                               dims=tuple(dims), state=st, params=p, far=True, child=child))
        self.set_outer_ghost(child, True)
        return len(self.blocks) - 1

    def far_step(self, i: int):
        """One step of far block i (its own dt = h dt_0) from t_n, linearly interpolated back
        to t_n + dt_0 (Sec. 4.2.4): f = (1 - 1/h) f(t_n) + (1/h) f(t_n + h dt_0); the stored
        velocity is recomputed from the interpolated populations, the scalar interpolated
        alike; obstacle and scale-boundary nodes keep their own values."""
        b = self.blocks[i]
        old = b.state
        new = grid.step(old, b.params)
        th = 1.0 / b.h
        f = (1.0 - th) * old.f + th * new.f
        c = (1.0 - th) * old.c + th * new.c
        _, u = cmr.macros(f.reshape(27, -1).T)
        u = u.T.reshape(old.u.shape)
        keep = (old.flags & (GHOST | SOLID | INFLOW)) != 0
        out = new.clone()
        out.f = torch.where(keep[None], new.f, f)
        out.u = torch.where(keep[None], new.u, u)
        out.c = torch.where(keep, new.c, c)
        b.state = out

    def far_out_map(self, i: int):
        """Scale-boundary nodes of far block i's child from block i (Sec. 4.2.5: the larger
        scale updates the boundary of the smaller one)."""
        b = self.blocks[i]
        c = self.blocks[b.child]
        z, y, x = self._ghost_nodes(c)
        f, cc, ok = interpolate(b, b.state.f, b.state.c, node_positions(c, z, y, x))
        c.state = rest_nodes(c.state, z[~ok], y[~ok], x[~ok])
        z, y, x, f, cc = z[ok], y[ok], x[ok], f[ok], cc[ok]
        fm = map_populations(f, k_hat(b, c))
        _, u = cmr.macros(fm)
        c.state = put_nodes(c.state, z, y, x, fm, u, cc)

    def _containing_parent(self, i: int) -> int:
        b = self.blocks[i]
        lo = b.origin
        hi = b.origin + (np.array(b.dims) - 1) * b.h
        best = 0
        for j in range(1, len(self.blocks)):
            c = self.blocks[j]
            if j == i or c.far or not c.h > b.h:
                continue
            clo = c.origin
            chi = c.origin + (np.array(c.dims) - 1) * c.h
            if np.all(clo <= lo + 1e-9) and np.all(hi <= chi + 1e-9):
                if c.h < self.blocks[best].h:
                    best = j
        return best

    # ------------------------------------------------------------------ mapping steps
    def _ghost_nodes(self, b: Blk):
        g = (b.state.flags & GHOST) != 0
        z, y, x = torch.nonzero(g, as_tuple=True)
        return z, y, x

    def prior_map(self, i: int, theta: float, saved: List[grid.State]):
        """Ghost layer of block i from its parent at time t_n + theta dt_0 (linear in time
        between the parent's state at t_n and its current state)."""
        b = self.blocks[i]
        p = self.blocks[b.parent]
        f_src = (1.0 - theta) * saved[b.parent].f + theta * p.state.f
        c_src = (1.0 - theta) * saved[b.parent].c + theta * p.state.c
        z, y, x = self._ghost_nodes(b)
        keep = (b.state.flags[z, y, x] & SOLID) == 0
        z, y, x = z[keep], y[keep], x[keep]
        f, c, ok = interpolate(p, f_src, c_src, node_positions(b, z, y, x))
        b.state = rest_nodes(b.state, z[~ok], y[~ok], x[~ok])
        z, y, x, f, c = z[ok], y[ok], x[ok], f[ok], c[ok]
        fm = map_populations(f, k_hat(p, b))
        _, u = cmr.macros(fm)
        b.state = put_nodes(b.state, z, y, x, fm, u, c)

    def post_map(self, i: int, k: int):
        """Coarser block k's nodes inside block i's interior span from block i."""
        b, tgt = self.blocks[i], self.blocks[k]
        lo, hi = b.interior_lo_hi()
        nx, ny, nz = tgt.dims
        zz, yy, xx = torch.meshgrid(torch.arange(nz), torch.arange(ny), torch.arange(nx),
                                    indexing="ij")
        pos = node_positions(tgt, zz.reshape(-1), yy.reshape(-1), xx.reshape(-1))
        eps = 1e-9
        inside = torch.ones(pos.shape[0], dtype=torch.bool)
        for a in range(3):
            inside &= (pos[:, a] >= lo[a] - eps) & (pos[:, a] <= hi[a] + eps)
        fl = tgt.state.flags.reshape(-1)
        inside &= (fl & (GHOST | SOLID)) == 0
        sel = torch.nonzero(inside).flatten()
        z, y, x = zz.reshape(-1)[sel], yy.reshape(-1)[sel], xx.reshape(-1)[sel]
        f, c, ok = interpolate(b, b.state.f, b.state.c, pos[sel])
        z, y, x, f, c = z[ok], y[ok], x[ok], f[ok], c[ok]
        fm = map_populations(f, k_hat(b, tgt))
        _, u = cmr.macros(fm)
        tgt.state = put_nodes(tgt.state, z, y, x, fm, u, c)

    @staticmethod
    def lagrange3(t0, t1, t2, T):
        L0 = (T - t1) * (T - t2) / ((t0 - t1) * (t0 - t2))
        L1 = (T - t0) * (T - t2) / ((t1 - t0) * (t1 - t2))
        L2 = (T - t0) * (T - t1) / ((t2 - t0) * (t2 - t1))
        return L0, L1, L2

    def align(self, b: Blk, s0: grid.State, s_prev: grid.State, s_last: grid.State):
        """Interior at t_n + dt_0 from the states at t_n, t_n+(l-1)h, t_n+l h."""
        l = b.substeps
        L0, L1, L2 = self.lagrange3(0.0, (l - 1) * b.h, l * b.h, 1.0)
        f = L0 * s0.f + L1 * s_prev.f + L2 * s_last.f
        c = L0 * s0.c + L1 * s_prev.c + L2 * s_last.c
        rho = f.sum(0)
        u = torch.einsum("qzyx,qa->azyx", f, cmr.C) / rho
        ghost = (b.state.flags & GHOST) != 0
        solid = (b.state.flags & SOLID) != 0
        if b.params.obstacle_walls:     # surface voxels are updated wall nodes: aligned too
            solid = solid & ~grid.surface_voxels(b.state.flags, b.params.periodic)
        keep = ghost | solid
        out = s_last.clone()
        out.f = torch.where(keep[None], s_last.f, f)
        out.u = torch.where(keep[None], s_last.u, u)
        out.c = torch.where(keep, s_last.c, c)
        return out

    # --------------------------------------------------------------------- Algorithm 1
    # One reference step, split into the phases a placement of blocks on several ranks
    # exchanges data between (begin, reference, per refined block its sub-cycle and its
    # post-mapping, end); step() runs them in order.
    def begin(self):
        self.saved = [b.state.clone() for b in self.blocks]

    def step_reference(self):
        """s0's step, then the far-field blocks' steps and their two mappings."""
        b0 = self.blocks[0]
        b0.state = grid.step(b0.state, b0.params)
        far = [i for i, b in enumerate(self.blocks) if b.far]
        for i in far:                      # far field: one own step, back to t_n + dt_0
            self.far_step(i)
        for i in far:                      # overlap of each far block from its child
            self.post_map(self.blocks[i].child, i)
        for i in reversed(far):            # scale boundary of each child from its far block
            self.far_out_map(i)

    def step_block(self, i):
        """Refined block i's sub-cycle: sub-steps with their scale boundaries, temporal
        alignment, and the scale boundary at t_n + dt_0."""
        b = self.blocks[i]
        saved = self.saved
        states = [b.state]
        for j in range(1, b.substeps + 1):
            self.prior_map(i, (j - 1) * b.h, saved)
            if j == 1:
                # the block's t_n state, with its ghost layer refreshed from the source
                # at t_n, is what finer blocks interpolate from
                saved[i] = b.state.clone()
            b.state = grid.step(b.state, b.params)
            states.append(b.state)
        if b.integer_ratio and abs(b.substeps * b.h - 1.0) < 1e-9:
            b.state = b.state.clone()
        else:
            prev = states[-2] if len(states) >= 2 else states[0]
            b.state = self.align(b, saved[i], prev, states[-1])
        self.prior_map(i, 1.0, saved)

    def post_block(self, i):
        """Post-mapping of refined block i into every coarser block."""
        b = self.blocks[i]
        for k in range(len(self.blocks)):
            if self.blocks[k].h > b.h and not self.blocks[k].far:
                self.post_map(i, k)

    def end(self):
        self.step_count += 1

    def step(self):
        self.begin()
        self.step_reference()
        for i in range(1, len(self.blocks)):
            if self.blocks[i].far:
                continue
            self.step_block(i)
            self.post_block(i)
        self.end()

    def run(self, n):
        for _ in range(n):
            self.step()
