"""FP64 reference for the non-orthogonal central-moment (CMR) collision on D3Q27.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``; never by the product path.

Everything here is the paper's definition written out with dense per-cell matrices and a
library LU solve; there is no factorisation, blocking or fusion.

Paper passages followed (arXiv 1807.02284, Li, Bai, Liu):
  * lattice velocities                           Appendix, velocity list (c_x, c_y, c_z)
  * central-moment matrix M_ij(u) = moment basis  Appendix, list of M_{i,0} .. M_{i,26};
    evaluated on translated velocities c - u      Sec. 3.1
  * m = M^T f, T = (M^T)^{-1}, f = T m            Sec. 3.1; Appendix
  * equilibrium central moments m^eq(rho, u)      Appendix, list m^eq_0 .. m^eq_26
  * collision Omega = -T S (m - m^eq)             Eq. (2) of Sec. 3.1 / Appendix
  * relaxation rates S_0..3 = 0, S_4..8 from nu,
    S_9..26 from the artificial viscosities nu'   Sec. 3.1, Eq. (3); Appendix
  * adaptive high-order viscosity                 Sec. 4.1 (adaptive relaxation equation)

Readings where the printed text is garbled (each pinned by a test):
  * The printed velocity list repeats (1,0,1) at index 13 and omits (1,0,-1); index 13 is
    read as (1,0,-1), the pattern of the neighbouring edge groups.
  * The printed M_{i,20} = cx^2 cy cz^2 duplicates M_{i,24} (M would be singular); it is
    read as cx^2 cy cz, the only third/fourth-order product missing from the list.
  * The index formula j = (m+1)(n+1)(p+1)-1 is not one-to-one; the explicit list is used.
  * The normalised gradient |grad u| / g_max is clamped to [0, 1] (g_max is the maximum
    gradient used for normalisation), so the viscosity factor stays in [a + b, b].
"""
from __future__ import annotations

import torch

DT = torch.float64

# Appendix: c_x, c_y, c_z of the 27 lattice velocities, as printed ...
PRINTED_CX = [0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1]
PRINTED_CY = [0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, 1, -1, -1, 1, 1, -1, -1]
PRINTED_CZ = [0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, 1, -1, 1, 1, -1, -1, 1, 1, 1, 1, -1, -1, -1, -1]
# ... with the duplicated entry at index 13 read as (1, 0, -1).
CZ_FIXED = list(PRINTED_CZ)
CZ_FIXED[13] = -1

C = torch.tensor([PRINTED_CX, PRINTED_CY, CZ_FIXED], dtype=DT).T.contiguous()  # (27, 3)
Q = 27


def _opposites():
    opp = []
    for i in range(Q):
        for j in range(Q):
            if torch.equal(C[j], -C[i]):
                opp.append(j)
                break
    return opp


OPP = _opposites()

# Appendix: artificial viscosities of the high-order groups (i = 9..16, 17..22, 23..25, 26)
NU_HI_DEFAULT = (0.005, 0.007, 0.009, 0.01)
# Sec. 4.1: adaptive-relaxation parameters
A_DEFAULT, B_DEFAULT = -4.0, 5.0
G_MAX_DEFAULT = 0.1       # low end of the printed range [0.1, 0.13]


def moment_matrix(u: torch.Tensor) -> torch.Tensor:
    """M(u)[..., i, j] = j-th central-moment basis function at translated velocity c_i - u.

    ``u`` has shape (..., 3); the result has shape (..., 27, 27).  Columns follow the
    Appendix list M_{i,0} .. M_{i,26} (with the M_{i,20} reading above).
    """
    cb = C - u[..., None, :]
    x, y, z = cb[..., 0], cb[..., 1], cb[..., 2]
    x2, y2, z2 = x * x, y * y, z * z
    cols = [
        torch.ones_like(x),            # 0
        x, y, z,                       # 1, 2, 3
        x * y, x * z, y * z,           # 4, 5, 6
        x2 - y2, x2 - z2,              # 7, 8
        x2 + y2 + z2,                  # 9
        x * y2 + x * z2,               # 10
        x2 * y + y * z2,               # 11
        x2 * z + y2 * z,               # 12
        x * y2 - x * z2,               # 13
        x2 * y - y * z2,               # 14
        x2 * z - y2 * z,               # 15
        x * y * z,                     # 16
        x2 * y2 + x2 * z2 + y2 * z2,   # 17
        x2 * y2 + x2 * z2 - y2 * z2,   # 18
        x2 * y2 - x2 * z2,             # 19
        x2 * y * z,                    # 20 (printed cx^2 cy cz^2; see module docstring)
        x * y2 * z,                    # 21
        x * y * z2,                    # 22
        x * y2 * z2,                   # 23
        x2 * y * z2,                   # 24
        x2 * y2 * z,                   # 25
        x2 * y2 * z2,                  # 26
    ]
    return torch.stack(cols, dim=-1)


def m_eq(rho: torch.Tensor, u: torch.Tensor) -> torch.Tensor:
    """Equilibrium central moments m^eq_0 .. m^eq_26 of the Appendix, shape (..., 27)."""
    ux, uy, uz = u[..., 0], u[..., 1], u[..., 2]
    x2, y2, z2 = ux * ux, uy * uy, uz * uz
    zero = torch.zeros_like(rho)
    r = rho
    vals = [
        r,                                                   # 0
        zero, zero, zero, zero, zero, zero, zero, zero,      # 1..8
        r,                                                   # 9
        -r * ux * (y2 + z2),                                 # 10
        -r * uy * (x2 + z2),                                 # 11
        -r * uz * (x2 + y2),                                 # 12
        -r * ux * (y2 - z2),                                 # 13
        -r * uy * (x2 - z2),                                 # 14
        -r * uz * (x2 - y2),                                 # 15
        -r * ux * uy * uz,                                   # 16
        r / 3.0 * (9 * x2 * y2 + 9 * x2 * z2 + 9 * y2 * z2 + 1),      # 17
        r / 9.0 * (27 * x2 * y2 + 27 * x2 * z2 - 27 * y2 * z2 + 1),   # 18
        3 * r * x2 * (y2 - z2),                              # 19
        3 * r * x2 * uy * uz,                                # 20
        3 * r * ux * y2 * uz,                                # 21
        3 * r * ux * uy * z2,                                # 22
        -r / 3.0 * ux * (18 * y2 * z2 + y2 + z2),            # 23
        -r / 3.0 * uy * (18 * x2 * z2 + x2 + z2),            # 24
        -r / 3.0 * uz * (18 * x2 * y2 + x2 + y2),            # 25
        r * (10 * x2 * y2 * z2 + x2 * y2 + x2 * z2 + y2 * z2 + 1.0 / 27.0),  # 26
    ]
    return torch.stack(vals, dim=-1)


def macros(f: torch.Tensor):
    """rho = sum_i f_i and u = sum_i c_i f_i / rho (Sec. 1, under the LBE)."""
    rho = f.sum(-1)
    u = (f @ C) / rho[..., None]
    return rho, u


def equilibrium(rho: torch.Tensor, u: torch.Tensor) -> torch.Tensor:
    """f = T m^eq(rho, u) with T = (M^T)^{-1}: the initial / Dirichlet state (Sec. 6.1)."""
    MT = moment_matrix(u).transpose(-1, -2)
    return torch.linalg.solve(MT, m_eq(rho, u)[..., None])[..., 0]


def relaxation_rates(nu: float, phi=None, nu_hi=NU_HI_DEFAULT, like=None) -> torch.Tensor:
    """Diagonal of S (Appendix): S_0..3 = 0; S_4..8 = 1/(3 nu + 1/2);
    S_i = 1/(3 phi nu'_i + 1/2) for i >= 9, with nu'_i from the four-group table and
    phi the adaptive factor of Sec. 4.1 (phi = 1 gives the fixed setting)."""
    if phi is None:
        phi = torch.ones((), dtype=DT) if like is None else torch.ones_like(like)
    phi = torch.as_tensor(phi, dtype=DT)
    S = [torch.zeros_like(phi)] * 4
    S += [torch.full_like(phi, 1.0 / (3.0 * nu + 0.5))] * 5
    groups = [(9, 17, nu_hi[0]), (17, 23, nu_hi[1]), (23, 26, nu_hi[2]), (26, 27, nu_hi[3])]
    for lo, hi, nup in groups:
        S += [1.0 / (3.0 * phi * nup + 0.5)] * (hi - lo)
    return torch.stack(S, dim=-1)


def adaptive_factor(grad_norm: torch.Tensor, a=A_DEFAULT, b=B_DEFAULT, g_max=G_MAX_DEFAULT):
    """Sec. 4.1: nu_hat'_i = (a |grad u| / g_max + b) nu'_i; returns the factor with the
    normalised gradient clamped to [0, 1]."""
    return a * torch.clamp(grad_norm / g_max, max=1.0) + b


def collide(f: torch.Tensor, S: torch.Tensor):
    """Post-collision state f~ = f + Omega, Omega = -T S (m - m^eq)  (Sec. 3.1).

    f: (..., 27), S: (..., 27) or (27,).  Returns (f~, rho, u) where rho and u are the
    macroscopic density and velocity of the pre-collision f (conserved by the collision).
    """
    rho, u = macros(f)
    M = moment_matrix(u)
    MT = M.transpose(-1, -2)
    m = (MT @ f[..., None])[..., 0]
    meq = m_eq(rho, u)
    m_star = m - S * (m - meq)
    f_post = torch.linalg.solve(MT, m_star[..., None])[..., 0]
    return f_post, rho, u
