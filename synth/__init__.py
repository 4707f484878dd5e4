"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and ``bench.py``.

This module holds *no* arithmetic of the solver: it only lays out geometry (voxelised
spheres, inflow disks), closed-form initial velocity fields of textbook test flows, and
seeded random numbers.  Both the FP64 oracle (``oracle/``) and the CUDA path receive
exactly these arrays, so any disagreement between them comes from the solver and not from
the inputs.

Conventions
-----------
* Arrays are indexed ``[z][y][x]``; vector fields are ``[3][z][y][x]`` with components
  ordered (x, y, z).
* Cell flags (uint8): ``SOLID`` obstacle voxel (halfway bounce-back), ``INFLOW`` Dirichlet
  equilibrium inflow, ``SCALAR_SRC`` passive-scalar source, ``GHOST`` scale-boundary node
  of a refined block (written only by the coarse-to-fine mapping).
* Velocities are lattice units of the block they live in.  Because every scale uses
  Δt = Δx, velocity is the same number on every scale (paper Sec. 4.2.4).

Workloads (shapes follow the paper's smoke and turbulence scenes, Sec. 6):
  ``taylor_green``   32^3 periodic decaying vortex (closed-form energy decay)
  ``plume``          256^3 inflow-disk smoke plume past a sphere
  ``multiscale``     3-block continuous-scale domain (h = 1, 1/1.5, 1/2.25)
  ``batch``          64 independent plumes with cube edges 24..96
  ``adjoint_scene``  128^3 periodic smoke-control problem (low-mode velocity + blobs)
  ``ringing_channel`` 196 x 98 x 98 flow past a sphere (relaxation comparison, Fig. 3)
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

SOLID = 1
INFLOW = 2
SCALAR_SRC = 4
GHOST = 8


@dataclasses.dataclass
class Block:
    """One uniform block of lattice nodes.

    ``origin`` is the position of node (0,0,0) in reference-scale units and ``h`` the node
    spacing relative to the reference scale (h = Δx_s / Δx_0).  Node k along an axis sits at
    ``origin + k*h``.
    """

    dims: Tuple[int, int, int]          # (nx, ny, nz)
    origin: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    h: float = 1.0
    flags: Optional[np.ndarray] = None  # uint8 [z][y][x]
    rho0: Optional[np.ndarray] = None   # float64 [z][y][x]
    u0: Optional[np.ndarray] = None     # float64 [3][z][y][x]; inflow cells hold u_in
    c0: Optional[np.ndarray] = None     # float64 [z][y][x]

    @property
    def shape_zyx(self):
        nx, ny, nz = self.dims
        return (nz, ny, nx)

    def node_coords(self):
        """Reference-unit coordinates of the nodes, each as a 1-D array per axis."""
        nx, ny, nz = self.dims
        ox, oy, oz = self.origin
        return (ox + self.h * np.arange(nx), oy + self.h * np.arange(ny),
                oz + self.h * np.arange(nz))


@dataclasses.dataclass
class Scene:
    blocks: List[Block]
    periodic: Tuple[bool, bool, bool]
    nu: float                     # kinematic viscosity in reference-scale lattice units
    adaptive: bool = True
    c_src: float = 1.0
    name: str = ""
    steps: int = 0


def _empty_block(dims, origin=(0.0, 0.0, 0.0), h=1.0) -> Block:
    nx, ny, nz = dims
    b = Block(dims=(nx, ny, nz), origin=tuple(float(o) for o in origin), h=float(h))
    b.flags = np.zeros((nz, ny, nx), np.uint8)
    b.rho0 = np.ones((nz, ny, nx), np.float64)
    b.u0 = np.zeros((3, nz, ny, nx), np.float64)
    b.c0 = np.zeros((nz, ny, nx), np.float64)
    return b


def voxelise_spheres(block: Block, spheres: Sequence[Tuple[float, float, float, float]]):
    """Mark nodes whose reference-unit position lies inside any (cx, cy, cz, r) sphere."""
    xs, ys, zs = block.node_coords()
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    for (cx, cy, cz, r) in spheres:
        inside = (X - cx) ** 2 + (Y - cy) ** 2 + (Z - cz) ** 2 <= r * r
        block.flags[inside] |= SOLID
    solid = (block.flags & SOLID) != 0
    block.u0[:, solid] = 0.0
    block.c0[solid] = 0.0


def inflow_disk(block: Block, center_yz, radius, u_in, rng=None, noise=0.0, scalar=True):
    """Flag an inflow disk on the x = 0 face; the inflow velocity is stored in ``u0``.

    ``noise`` adds seeded uniform +/- noise (relative) per cell and component, fixed in time.
    """
    nx, ny, nz = block.dims
    ys = np.arange(ny)
    zs = np.arange(nz)
    Z, Y = np.meshgrid(zs, ys, indexing="ij")
    disk = (Y - center_yz[0]) ** 2 + (Z - center_yz[1]) ** 2 <= radius * radius
    zi, yi = np.nonzero(disk)
    vel = np.zeros((3, zi.size))
    vel[0] = u_in
    if noise > 0.0:
        vel = vel + noise * abs(u_in) * (2.0 * rng.random((3, zi.size)) - 1.0)
    block.flags[zi, yi, 0] |= INFLOW
    block.flags[zi, yi, 0] &= np.uint8(~SOLID & 0xFF)
    block.u0[:, zi, yi, 0] = vel
    if scalar:
        block.flags[zi, yi, 0] |= SCALAR_SRC
        block.c0[zi, yi, 0] = 1.0
    return zi, yi, vel


def inflow_records(block: Block) -> np.ndarray:
    """Inflow cells as int32/float32 records ``(x, y, z, ux, uy, uz)`` for the C-ABI."""
    z, y, x = np.nonzero(block.flags & INFLOW)
    rec = np.zeros(z.size, dtype=[("x", "<i4"), ("y", "<i4"), ("z", "<i4"),
                                  ("ux", "<f4"), ("uy", "<f4"), ("uz", "<f4")])
    rec["x"], rec["y"], rec["z"] = x, y, z
    rec["ux"], rec["uy"], rec["uz"] = (block.u0[0, z, y, x], block.u0[1, z, y, x],
                                      block.u0[2, z, y, x])
    return rec


# --------------------------------------------------------------------------- workloads

def taylor_green(n=32, u0=0.05, nz=None, re=100.0, adaptive=True) -> Scene:
    """z-invariant Taylor-Green vortex on an n x n x nz periodic box.

    u = u0 sin(kx) cos(ky), v = -u0 cos(kx) sin(ky), w = 0 with k = 2 pi / n and the matching
    pressure rho = 1 - (3 u0^2 / 4)(cos 2kx + cos 2ky).  nu = u0 n / Re.
    """
    nz = n if nz is None else nz
    b = _empty_block((n, n, nz))
    k = 2.0 * math.pi / n
    x = np.arange(n)[None, None, :]
    y = np.arange(n)[None, :, None]
    shape = (nz, n, n)
    b.u0[0] = np.broadcast_to(u0 * np.sin(k * x) * np.cos(k * y), shape)
    b.u0[1] = np.broadcast_to(-u0 * np.cos(k * x) * np.sin(k * y), shape)
    b.rho0[:] = np.broadcast_to(1.0 - 0.75 * u0 * u0 * (np.cos(2 * k * x) + np.cos(2 * k * y)),
                                shape)
    return Scene(blocks=[b], periodic=(True, True, True), nu=u0 * n / re, adaptive=adaptive,
                 name=f"taylor_green_{n}x{n}x{nz}")


def taylor_green_3d(n=32, u0=0.05, re=100.0) -> Scene:
    """Classical 3-D Taylor-Green initial field (no closed form; used for parity only)."""
    b = _empty_block((n, n, n))
    k = 2.0 * math.pi / n
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    b.u0[0] = u0 * np.sin(k * x) * np.cos(k * y) * np.cos(k * z)
    b.u0[1] = -u0 * np.cos(k * x) * np.sin(k * y) * np.cos(k * z)
    b.rho0[:] = 1.0
    return Scene(blocks=[b], periodic=(True, True, True), nu=u0 * n / re,
                 name=f"taylor_green_3d_{n}")


def random_velocity(shape_zyx, seed, amp=0.05, kmax=3, periodic=True) -> np.ndarray:
    """Seeded smooth velocity field: a sum of low Fourier modes (|k_i| <= kmax), max |u| = amp."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape_zyx
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    u = np.zeros((3,) + tuple(shape_zyx))
    for a in range(3):
        for _ in range(6):
            kx, ky, kz = rng.integers(-kmax, kmax + 1, size=3)
            ph = rng.random() * 2 * math.pi
            amp_m = rng.standard_normal()
            u[a] += amp_m * np.cos(2 * math.pi * (kx * x / nx + ky * y / ny + kz * z / nz) + ph)
    m = np.abs(u).max()
    if m > 0:
        u *= amp / m
    return u


def random_scene(dims=(20, 18, 16), seed=0, periodic=(True, True, True), nu=0.02,
                 spheres=(), inflow=None, adaptive=True, amp=0.05) -> Scene:
    """Small seeded scene for parity tests: smooth random velocity, optional obstacles
    and inflow disk, random density perturbation and a random scalar field."""
    rng = np.random.default_rng(seed)
    b = _empty_block(dims)
    b.u0[:] = random_velocity(b.shape_zyx, seed + 1000, amp=amp)
    b.rho0[:] = 1.0 + 0.01 * (2 * rng.random(b.shape_zyx) - 1)
    b.c0[:] = rng.random(b.shape_zyx)
    if spheres:
        voxelise_spheres(b, spheres)
    if inflow is not None:
        cy, cz, r, u_in = inflow
        inflow_disk(b, (cy, cz), r, u_in, rng=rng, noise=0.01)
    solid = (b.flags & SOLID) != 0
    b.rho0[solid] = 1.0
    return Scene(blocks=[b], periodic=tuple(periodic), nu=nu, adaptive=adaptive,
                 name=f"random_{dims}_{seed}")


def random_populations(shape_zyx, seed, base=None, eps=0.02) -> np.ndarray:
    """Seeded positive populations f[27][z][y][x] = base_q (1 + eps r), r uniform in [-1, 1].

    ``base`` defaults to a fixed positive per-direction profile (rest 0.3, faces 0.07,
    edges 0.02, corners 0.005); the values are only plausible magnitudes, not an equilibrium.
    """
    rng = np.random.default_rng(seed)
    if base is None:
        base = np.array([0.3] + [0.07] * 6 + [0.02] * 12 + [0.005] * 8)
        # order of the paper's velocity list: rest, 6 faces, 12 edges, 8 corners
    r = 2.0 * rng.random((27,) + tuple(shape_zyx)) - 1.0
    return base[:, None, None, None] * (1.0 + eps * r)


def plume(n=256, seed=1, nu=1e-5, u_in=0.1, r_in=16, sphere_r=24) -> Scene:
    """Smoke plume: inflow disk (radius r_in, +/-1% seeded noise) on the x=0 face, a
    voxelised sphere of radius sphere_r at (72, n/2, n/2) (scaled with n), Neumann faces."""
    rng = np.random.default_rng(seed)
    s = n / 256.0
    b = _empty_block((n, n, n))
    inflow_disk(b, (n / 2, n / 2), r_in * s, u_in, rng=rng, noise=0.01)
    voxelise_spheres(b, [(72 * s, n / 2, n / 2, sphere_r * s)])
    return Scene(blocks=[b], periodic=(False, False, False), nu=nu, adaptive=True,
                 name=f"plume_{n}", steps=1000)


def ringing_channel(seed=6, nu=1e-4, u_in=0.1, r_in=12, sphere_r=12) -> Scene:
    """Flow past a sphere in a 196 x 98 x 98 box with nu = 1e-4, the resolution and viscosity
    of the relaxation comparison of Fig. 3: inflow disk (radius r_in, +/-1% seeded noise) on
    the x = 0 face, a voxelised sphere at (40, 49, 49), Neumann faces."""
    rng = np.random.default_rng(seed)
    b = _empty_block((196, 98, 98))
    inflow_disk(b, (49.0, 49.0), r_in, u_in, rng=rng, noise=0.01)
    voxelise_spheres(b, [(40.0, 49.0, 49.0, sphere_r)])
    return Scene(blocks=[b], periodic=(False, False, False), nu=nu, adaptive=True,
                 name="ringing_196", steps=2000)


def smooth_field(block: Block, seed, amp=0.05, wavelength=32.0):
    """Seeded sum of low Fourier modes evaluated at the block's node positions (reference
    units), so overlapping blocks of any spacing sample the same continuous field.
    Returns (u (3,z,y,x), rho (z,y,x), c (z,y,x))."""
    rng = np.random.default_rng(seed)
    xs, ys, zs = block.node_coords()
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    k = 2 * math.pi / wavelength
    u = np.zeros((3,) + Z.shape)
    for a in range(3):
        for _ in range(3):
            kv = rng.integers(-2, 3, size=3)
            ph = rng.random() * 2 * math.pi
            u[a] += rng.standard_normal() * np.cos(k * (kv[0] * X + kv[1] * Y + kv[2] * Z) + ph)
    m = max(np.abs(u).max(), 1e-12)
    u *= amp / m
    rho = 1.0 + 0.2 * amp * np.cos(k * (X + 2 * Y - Z) + rng.random())
    c = 0.5 + 0.5 * np.sin(k * (2 * X - Y) + rng.random()) * np.cos(k * Z)
    return u, rho, c


def far_block(inner: Block, h: float, pad: float, seed=0, amp=0.02, wavelength=32.0) -> Block:
    """A far-field block of spacing h (> 1) around ``inner``: it starts ``pad`` reference
    units below inner's lower corner on every axis and reaches at least ``pad`` beyond its
    upper corner; seeded smooth velocity, density and scalar fields (the same continuous
    fields on any block), no obstacles."""
    lo = np.array(inner.origin, dtype=np.float64) - pad
    hi = np.array(inner.origin, dtype=np.float64) + (np.array(inner.dims) - 1) * inner.h + pad
    dims = tuple(int(math.ceil((hi[a] - lo[a]) / h - 1e-9)) + 1 for a in range(3))
    b = _empty_block(dims, origin=tuple(lo), h=h)
    u, rho, c = smooth_field(b, seed, amp=amp, wavelength=wavelength)
    b.u0, b.rho0, b.c0 = u, rho, c
    return b


def multiscale(seed=2, sphere_seed=3, nu=1e-5, u_in=0.08, scale=1.0, flow_amp=0.0) -> Scene:
    """Continuous-scale 3-block domain: s0 128^3 at h=1, s1 96^3 at h=1/1.5 with origin
    (24,32,32), s2 64^3 at h=1/2.25 with origin (36,50,50); 8 seeded spheres (r in [4,12])
    inside s1's span; inflow at x=0 of s0 with +/-1% noise.  ``scale`` < 1 shrinks every
    length (block edges, origins, radii) for oracle-sized copies."""
    rng = np.random.default_rng(seed)
    srng = np.random.default_rng(sphere_seed)
    n0 = max(8, int(round(128 * scale)))
    n1 = max(8, int(round(96 * scale)))
    n2 = max(8, int(round(64 * scale)))
    s0 = _empty_block((n0, n0, n0))
    s1 = _empty_block((n1, n1, n1), origin=(24 * scale, 32 * scale, 32 * scale), h=1 / 1.5)
    s2 = _empty_block((n2, n2, n2), origin=(36 * scale, 50 * scale, 50 * scale), h=1 / 2.25)
    lo = np.array(s1.origin)
    span = (n1 - 1) * s1.h
    spheres = []
    for _ in range(8):
        r = (4 + 8 * srng.random()) * scale
        c = lo + span * (0.15 + 0.7 * srng.random(3))
        spheres.append((float(c[0]), float(c[1]), float(c[2]), float(r)))
    if flow_amp > 0.0:
        for b in (s0, s1, s2):
            b.u0[:], b.rho0[:], b.c0[:] = smooth_field(b, seed + 100, amp=flow_amp,
                                                      wavelength=max(8.0, 32.0 * scale))
    inflow_disk(s0, (n0 / 2, n0 / 2), 0.25 * n0, u_in, rng=rng, noise=0.01)
    for b in (s0, s1, s2):
        voxelise_spheres(b, spheres)
        b.rho0[(b.flags & SOLID) != 0] = 1.0
    return Scene(blocks=[s0, s1, s2], periodic=(False, False, False), nu=nu, adaptive=True,
                 name=f"multiscale_{n0}_{n1}_{n2}", steps=500)


def batch(count=64, seed=4, lo=24, hi=96, nu=1e-5) -> List[Scene]:
    """Independent plumes with cube edge L ~ U{lo..hi}, 1-4 spheres of radius U[2, L/8]
    and inflow speed U[0.03, 0.1]."""
    rng = np.random.default_rng(seed)
    scenes = []
    for i in range(count):
        L = int(rng.integers(lo, hi + 1))
        b = _empty_block((L, L, L))
        u_in = float(rng.uniform(0.03, 0.1))
        inflow_disk(b, (L / 2, L / 2), max(2.0, L / 8), u_in, rng=rng, noise=0.01)
        k = int(rng.integers(1, 5))
        sph = []
        for _ in range(k):
            r = float(rng.uniform(2, max(2.0, L / 8)))
            c = rng.uniform(0.3 * L, 0.8 * L, size=3)
            sph.append((float(c[0]), float(c[1]), float(c[2]), r))
        voxelise_spheres(b, sph)
        scenes.append(Scene(blocks=[b], periodic=(False, False, False), nu=nu,
                            name=f"batch_{i}_{L}", steps=300))
    return scenes


def gaussian_blob(shape_zyx, center_xyz, sigma) -> np.ndarray:
    nz, ny, nx = shape_zyx
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cx, cy, cz = center_xyz
    return np.exp(-((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2) / (2.0 * sigma * sigma))


def adjoint_scene(n=128, seed=5, nu=1e-3, amp=0.05, steps=200):
    """Smoke-control problem: periodic n^3 box, low-mode seeded velocity (|k| <= 4 scaled to
    the box), scalar Gaussian blob (sigma = n/16) at the centre, and a target blob of the same
    width offset by a seeded vector with |d| <= n/16.  Returns (scene, target)."""
    rng = np.random.default_rng(seed)
    b = _empty_block((n, n, n))
    b.u0[:] = random_velocity(b.shape_zyx, seed + 77, amp=amp, kmax=max(1, min(4, n // 8)))
    sig = n / 16.0
    ctr = (n / 2.0, n / 2.0, n / 2.0)
    b.c0[:] = gaussian_blob(b.shape_zyx, ctr, sig)
    d = rng.standard_normal(3)
    d *= (n / 16.0) * rng.random() / max(np.linalg.norm(d), 1e-12)
    target = gaussian_blob(b.shape_zyx, tuple(np.array(ctr) + d), sig)
    sc = Scene(blocks=[b], periodic=(True, True, True), nu=nu, adaptive=True,
               name=f"adjoint_{n}", steps=steps)
    return sc, target
