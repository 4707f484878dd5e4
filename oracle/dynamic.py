"""Dynamic scale construction (Sec. 5) — test infrastructure, never part of the product path.

Plain FP64 restatement of how a dynamic scale is found, placed and started:

  1. detection (Sec. 5): on a block's stored velocity field, keep the samples whose gradient
     magnitude is at least g_threshold, then of those the samples whose velocity magnitude is
     at least u_threshold; what remains is one dynamic-scale region;
  2. placement: the region becomes a box block of spacing h;
  3. start: the new block's samples are mapped from the coarser scale it is overlaid on
     (Sec. 3.2 mapping with K_hat, at the current time), after any previous dynamic scale
     has been discarded.

Readings (the paper describes the procedure in words only):
  * The gradient magnitude is the Frobenius norm of the central-difference Jacobian of the
    stored velocity, the quantity the adaptive factor uses (grid.lagged_gradient_norm), in
    the detection block's lattice units; the velocity magnitude is |u|.  Obstacle voxels and
    ghost nodes are never selected.  The two thresholds applied one after the other select
    the same samples as their conjunction.
  * The region is represented by its axis-aligned bounding box in the detection block's node
    indices, widened by `margin` of those nodes on every side and clipped to the reference
    block [0, n_0 - 1] (reference units).  The new block starts at the clipped lower corner;
    it has floor(extent / h + 1e-9) + 1 nodes per axis, at least 4, shifted down (not below
    0) when 4 nodes would pass the reference block's upper end.
  * Obstacle and scalar-source bits of the new block come from the nearest node of its
    prior-mapping source (index floor(q + 1/2) of the node's position q in that block's node
    units, clamped to the block); its outermost layer is its ghost layer.  (With the
    reference block as detection block and source, as in the paper's jet flows, the two
    are the same block.)
  * Every non-obstacle node of the new block, ghost layer included, is set to the mapping of
    its prior-mapping source (the finest coarser block containing it) at the current time;
    its velocity is that of the mapped populations and its scalar is interpolated.  Obstacle
    nodes hold the rest state.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import cmr, coupling, grid

SOLID, INFLOW, SCALAR_SRC, GHOST = grid.SOLID, grid.INFLOW, grid.SCALAR_SRC, grid.GHOST


def detect(state: grid.State, periodic, g_threshold: float, u_threshold: float):
    """(count, box) of the selected samples; box = (x0, y0, z0, x1, y1, z1) inclusive node
    indices, or None when nothing is selected.  Also returns the per-node gradient and
    velocity magnitudes (for tie checks in tests)."""
    _, Z, Y, X = state.u.shape
    z, y, x = torch.meshgrid(torch.arange(Z), torch.arange(Y), torch.arange(X), indexing="ij")
    g = grid.lagged_gradient_norm(state.u, periodic, z, y, x)
    umag = torch.sqrt((state.u ** 2).sum(0))
    excluded = (state.flags & (SOLID | GHOST)) != 0
    keep = (g >= g_threshold) & ~excluded          # first threshold: gradient magnitude
    keep = keep & (umag >= u_threshold)             # second threshold: velocity magnitude
    n = int(keep.sum())
    if n == 0:
        return 0, None, g, umag
    zz, yy, xx = torch.nonzero(keep, as_tuple=True)
    box = (int(xx.min()), int(yy.min()), int(zz.min()), int(xx.max()), int(yy.max()), int(zz.max()))
    return n, box, g, umag


def place(box, src_origin, src_h: float, h: float, margin: int, ref_dims):
    """Origin (reference units) and node counts of the dynamic block for a detection box of
    a block with origin src_origin and spacing src_h."""
    origin, dims = [], []
    for a in range(3):
        lo = src_origin[a] + (box[a] - margin) * src_h
        hi = src_origin[a] + (box[3 + a] + margin) * src_h
        top = float(ref_dims[a] - 1)
        lo = max(lo, 0.0)
        hi = min(hi, top)
        n = max(int(math.floor((hi - lo) / h + 1e-9)) + 1, 4)
        if lo + (n - 1) * h > top + 1e-9:
            lo = max(0.0, top - (n - 1) * h)
        origin.append(lo)
        dims.append(n)
    return tuple(origin), tuple(dims)


def nearest_flags(src: coupling.Blk, origin, h: float, dims):
    """Obstacle / scalar-source bits of a new block from the nearest source node, plus its
    ghost layer.  Returns uint8 flags shaped (z, y, x)."""
    nx, ny, nz = dims
    idx = []
    for a, n in enumerate((nx, ny, nz)):
        q = (origin[a] + h * np.arange(n) - src.origin[a]) / src.h
        i = np.clip(np.floor(q + 0.5).astype(np.int64), 0, src.dims[a] - 1)
        idx.append(i)
    sf = src.state.flags.numpy()
    fl = sf[np.ix_(idx[2], idx[1], idx[0])] & (SOLID | SCALAR_SRC)
    fl = fl.astype(np.uint8)
    fl[0, :, :] |= GHOST
    fl[-1, :, :] |= GHOST
    fl[:, 0, :] |= GHOST
    fl[:, -1, :] |= GHOST
    fl[:, :, 0] |= GHOST
    fl[:, :, -1] |= GHOST
    return fl


def add_block_from_parent(ms: coupling.MultiScale, origin, h: float, dims):
    """Appends a dynamic block to a MultiScale domain and starts it from its parent (the
    finest coarser block containing it), which also gives its obstacle / source bits."""
    nx, ny, nz = dims
    ref = ms.blocks[0].params
    nu_b = ref.nu / h
    p = grid.Params(nu=nu_b, periodic=(False, False, False), adaptive=ref.adaptive,
                    c_src=ref.c_src, grad_mode=ref.grad_mode)
    ratio = 1.0 / h
    zeros = np.zeros((nz, ny, nx))
    st = grid.init_state(np.ones((nz, ny, nx)), np.zeros((3, nz, ny, nx)), zeros,
                         np.zeros((nz, ny, nx), np.uint8))
    b = coupling.Blk(origin=np.array(origin, dtype=np.float64), h=float(h), dims=tuple(dims),
                     state=st, params=p, substeps=max(1, math.ceil(ratio - 1e-9)),
                     integer_ratio=abs(ratio - round(ratio)) < 1e-9)
    ms.blocks.append(b)
    i = len(ms.blocks) - 1
    b.parent = ms._containing_parent(i)
    par = ms.blocks[b.parent]
    flags = torch.as_tensor(nearest_flags(par, origin, h, dims))
    st = grid.init_state(np.ones((nz, ny, nx)), np.zeros((3, nz, ny, nx)), zeros, flags)
    b.state = st
    z, y, x = torch.nonzero((st.flags & SOLID) == 0, as_tuple=True)
    f, c, ok = coupling.interpolate(par, par.state.f, par.state.c,
                                    coupling.node_positions(b, z, y, x))
    z, y, x, f, c = z[ok], y[ok], x[ok], f[ok], c[ok]
    fm = coupling.map_populations(f, coupling.k_hat(par, b))
    _, u = cmr.macros(fm)
    b.state = coupling.put_nodes(st, z, y, x, fm, u, c)
    return i


def remove_last_block(ms: coupling.MultiScale):
    """Discards the most recently added block (its interior was post-mapped into every
    coarser block at the end of each reference step)."""
    if len(ms.blocks) < 2:
        raise ValueError("only refined blocks can be removed")
    ms.blocks.pop()


# ------------------------------------------------------------------ static construction

def obstacle_box(flags):
    """Bounding box (x0, y0, z0, x1, y1, z1) of the obstacle voxels of a block, or None."""
    zz, yy, xx = np.nonzero((np.asarray(flags) & SOLID) != 0)
    if zz.size == 0:
        return None
    return (int(xx.min()), int(yy.min()), int(zz.min()), int(xx.max()), int(yy.max()), int(zz.max()))


def static_scales(flags, n_scales: int, h_min: float, d_max: float, wake: float, flow_axis: int = 0):
    """Static scale construction (Sec. 5) on the reference block: the distance to the
    obstacles is quantised into n_scales scales, scale 0 being s0 (h = 1) and scale
    n_scales - 1 the finest (h = h_min), the spacings linearly interpolated in between.
    Scale i covers the samples within d_i = d_max (n - 1 - i) / (n - 1) of an obstacle,
    extended downstream along flow_axis by `wake` (the wake region behind the object).

    Readings: blocks are boxes, and the bounding box of the samples within d of the
    obstacles is the obstacles' bounding box widened by d; the wake extension is the same
    for every refined scale; each box is clipped to s0, snapped to the finest whole number of
    its own spacing inside the clipped span, and kept at >= 4 nodes per axis (growing upward,
    or shifted down at s0's upper end).  Returns [(origin, h, dims)] for scales 1 .. n-1,
    coarse to fine (empty without obstacles)."""
    box = obstacle_box(flags)
    if box is None or n_scales < 2:
        return []
    Z, Y, X = np.asarray(flags).shape
    ref = (X, Y, Z)
    out = []
    for i in range(1, n_scales):
        h = 1.0 + (h_min - 1.0) * i / (n_scales - 1)
        d = d_max * (n_scales - 1 - i) / (n_scales - 1)
        lo = [box[a] - d for a in range(3)]
        hi = [box[3 + a] + d for a in range(3)]
        hi[flow_axis] += wake
        origin, dims = [], []
        for a in range(3):
            top = float(ref[a] - 1)
            l, u = max(lo[a], 0.0), min(hi[a], top)
            n = max(int(math.floor((u - l) / h + 1e-9)) + 1, 4)
            if l + (n - 1) * h > top + 1e-9:
                l = max(0.0, top - (n - 1) * h)
            origin.append(l)
            dims.append(n)
        out.append((tuple(origin), h, tuple(dims)))
    return out


# ------------------------------------------------------------- soft-shadow wake (Sec. 5)

def light_samples(flags, flow_axis: int, n_light: int):
    """Points of the inlet taken as the area light source: the inflow nodes (in index order,
    every ceil(count / n_light)-th one), or, without inflow nodes, the nodes of the upstream
    face (index 0 along flow_axis) the same way.  Returns an (M, 3) int array of (x, y, z)."""
    f = np.asarray(flags)
    z, y, x = np.nonzero((f & INFLOW) != 0)
    if z.size == 0:
        Z, Y, X = f.shape
        face = np.zeros_like(f, dtype=bool)
        sl = [slice(None)] * 3
        sl[2 - flow_axis] = 0
        face[tuple(sl)] = True
        z, y, x = np.nonzero(face)
    stride = -(-z.size // n_light)
    return np.stack([x, y, z], 1)[::stride]


def visibility(flags, nodes, lights):
    """Number of light samples each node (K, 3 ints x, y, z) sees: the straight segment from
    the node to the sample crosses no obstacle voxel.  The segment is walked in 2 m steps, m
    the largest coordinate difference; step k sits at p + d k / (2 m) and is checked at its
    nearest voxel, floor(q + 1/2), all in integer arithmetic (the two end points are not
    checked)."""
    f = np.asarray(flags)
    solid = (f & SOLID) != 0
    nodes = np.asarray(nodes, np.int64)
    count = np.zeros(len(nodes), np.int64)
    for L in np.asarray(lights, np.int64):
        d = L[None, :] - nodes
        m = np.abs(d).max(1)
        n = 2 * m
        blocked = np.zeros(len(nodes), bool)
        for k in range(1, int(n.max(initial=0))):
            act = np.nonzero(k < n)[0]
            if act.size == 0:
                break
            na = n[act][:, None]
            v = (2 * (nodes[act] * na + d[act] * k) + na) // (2 * na)
            blocked[act] |= solid[v[:, 2], v[:, 1], v[:, 0]]
        count += ~blocked
    return count


def shadow_scales(flags, n_scales: int, h_min: float, d_max: float, wake: float,
                  flow_axis: int = 0, n_light: int = 16):
    """Static scale construction with the wake shaped like a soft shadow (Sec. 5): the inlet
    is an area light source (light_samples); a node downstream of the obstacles (from the
    obstacles' upstream end to `wake` past their downstream end along flow_axis, obstacle
    voxels excluded) that sees c of the M samples belongs to the wake of scale i (i = 1 .. n-1,
    coarse to fine) when c (n - 1) <= (n - 1 - i) M: the finest scale takes the umbra (c = 0),
    coarser ones more and more of the penumbra.  Scale i covers the obstacles' box widened by
    d_i (as in static_scales) together with the bounding box of its wake nodes, clipped and
    snapped like static_scales.  Returns [(origin, h, dims)] for scales 1 .. n-1."""
    box = obstacle_box(flags)
    if box is None or n_scales < 2:
        return []
    f = np.asarray(flags)
    Z, Y, X = f.shape
    ref = (X, Y, Z)
    lights = light_samples(f, flow_axis, n_light)
    M = len(lights)
    lo_a = int(box[flow_axis])
    hi_a = int(min(math.floor(box[3 + flow_axis] + wake), ref[flow_axis] - 1))
    zz, yy, xx = np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    coord = (xx, yy, zz)
    cand = (coord[flow_axis] >= lo_a) & (coord[flow_axis] <= hi_a) & ((f & SOLID) == 0)
    zi, yi, xi = np.nonzero(cand)
    nodes = np.stack([xi, yi, zi], 1)
    c = visibility(f, nodes, lights)
    out = []
    for i in range(1, n_scales):
        h = 1.0 + (h_min - 1.0) * i / (n_scales - 1)
        d = d_max * (n_scales - 1 - i) / (n_scales - 1)
        lo = [box[a] - d for a in range(3)]
        hi = [box[3 + a] + d for a in range(3)]
        sel = c * (n_scales - 1) <= (n_scales - 1 - i) * M
        if sel.any():
            for a in range(3):
                lo[a] = min(lo[a], float(nodes[sel, a].min()))
                hi[a] = max(hi[a], float(nodes[sel, a].max()))
        origin, dims = [], []
        for a in range(3):
            top = float(ref[a] - 1)
            l, u = max(lo[a], 0.0), min(hi[a], top)
            n = max(int(math.floor((u - l) / h + 1e-9)) + 1, 4)
            if l + (n - 1) * h > top + 1e-9:
                l = max(0.0, top - (n - 1) * h)
            origin.append(l)
            dims.append(n)
        out.append((tuple(origin), h, tuple(dims)))
    return out
