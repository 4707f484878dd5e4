"""FP64 gradients of a smoke-control loss with respect to the initial velocity field.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper has no adjoint; this module differentiates the oracle's own forward model
(``oracle.grid``: equilibrium initialisation, pull, bounce-back, CMR collision with the
adaptive rates, semi-Lagrangian scalar) in reverse mode with torch's autograd, in float64,
recomputing each step during the backward sweep (per-step checkpoints) to bound memory.
It is itself checked against central finite differences of the same forward model.

Loss: L = 1/2 sum_x (c_T(x) - c_target(x))^2 (+ optional 1/2 sum |u_T - u_target|^2).
"""
from __future__ import annotations

import numpy as np
import torch
from torch.utils.checkpoint import checkpoint

from . import cmr, grid
from .cmr import DT


def _step_tensors(f, u, c, flags, p):
    st = grid.step(grid.State(f, u, c, flags), p)
    return st.f, st.u, st.c


def forward(u0: torch.Tensor, rho0, c0, flags, p: grid.Params, steps: int,
            use_checkpoint: bool = True, restart=None):
    """Runs `steps` steps from the equilibrium of (rho0, u0); returns the final State.

    ``restart`` (optional) maps step numbers n to states (f, u, c): at the start of step n
    the running state takes those values while its derivative passes through unchanged
    (straight-through), which is how a reverse sweep that replays each segment from a stored
    checkpoint sees a forward whose stored states were rounded (FP16-shifted storage)."""
    flags_t = torch.as_tensor(np.asarray(flags).astype(np.uint8)) \
        if not isinstance(flags, torch.Tensor) else flags
    st = grid.init_state(torch.as_tensor(np.asarray(rho0), dtype=DT), u0,
                         torch.as_tensor(np.asarray(c0), dtype=DT), flags_t)
    f, u, c = st.f, st.u, st.c
    for n in range(steps):
        if restart is not None and n in restart:
            rf, ru, rc = restart[n]
            f = f + (rf - f).detach()
            u = u + (ru - u).detach()
            c = c + (rc - c).detach()
        if use_checkpoint and torch.is_grad_enabled():
            f, u, c = checkpoint(_step_tensors, f, u, c, flags_t, p, use_reentrant=False)
        else:
            f, u, c = _step_tensors(f, u, c, flags_t, p)
    return grid.State(f, u, c, flags_t)


def round_shifted_to_half(f: torch.Tensor) -> torch.Tensor:
    """FP16-shifted storage of populations (27, ...): the deviation d = f - w from the lattice
    weights rounded to binary16 (round to nearest even), then widened back."""
    w = cmr.equilibrium(torch.ones(1, dtype=DT), torch.zeros(1, 3, dtype=DT))[0]
    w = w.reshape((27,) + (1,) * (f.dim() - 1))
    return (f - w).to(torch.float16).to(DT) + w


def fp16_storage_checkpoints(u0, rho0, c0, flags, p: grid.Params, steps: int, every: int):
    """States of the FP16-shifted-storage forward (the deviations rounded to binary16 after
    the initialisation and after every step; velocity and scalar kept in full precision) at
    every multiple of `every` below `steps`: the checkpoints a reverse sweep replays from."""
    with torch.no_grad():
        flags_t = torch.as_tensor(np.asarray(flags).astype(np.uint8))
        st = grid.init_state(torch.as_tensor(np.asarray(rho0), dtype=DT),
                             torch.as_tensor(np.asarray(u0), dtype=DT),
                             torch.as_tensor(np.asarray(c0), dtype=DT), flags_t)
        st.f = round_shifted_to_half(st.f)
        out = {}
        for n in range(steps):
            if n % every == 0:
                out[n] = (st.f.clone(), st.u.clone(), st.c.clone())
            st = grid.step(st, p)
            st.f = round_shifted_to_half(st.f)
        return out


def loss_fn(st: grid.State, c_target, u_target=None):
    L = 0.5 * ((st.c - torch.as_tensor(np.asarray(c_target), dtype=DT)) ** 2).sum()
    if u_target is not None:
        L = L + 0.5 * ((st.u - torch.as_tensor(np.asarray(u_target), dtype=DT)) ** 2).sum()
    return L


def loss_and_grad(u0, rho0, c0, flags, p: grid.Params, steps: int, c_target, u_target=None,
                  restart=None):
    """(L, dL/du0, c_T) in float64 (``restart``: see ``forward``)."""
    u = torch.as_tensor(np.asarray(u0), dtype=DT).clone().requires_grad_(True)
    st = forward(u, rho0, c0, flags, p, steps, restart=restart)
    L = loss_fn(st, c_target, u_target)
    (g,) = torch.autograd.grad(L, u)
    return float(L.detach()), g.detach(), st.c.detach()


def loss_only(u0, rho0, c0, flags, p: grid.Params, steps: int, c_target, u_target=None):
    with torch.no_grad():
        u = torch.as_tensor(np.asarray(u0), dtype=DT)
        st = forward(u, rho0, c0, flags, p, steps, use_checkpoint=False)
        return float(loss_fn(st, c_target, u_target))


# ---------------------------------------------------------------- continuous-scale domains

def ms_forward(scene, u0s, steps: int, f32_inputs=True, far=()):
    """Runs a continuous-scale domain (oracle.coupling.MultiScale: s0, refined blocks, and
    the far-field blocks `far` (synth Blocks, h > 1) added in order after them) from the
    equilibria of (rho0_b, u0s[b]) for `steps` reference steps; returns it."""
    from . import coupling
    ms = coupling.MultiScale.build(scene, f32_inputs=f32_inputs)
    conv = (lambda a: torch.as_tensor(np.asarray(a, np.float32).astype(np.float64))) \
        if f32_inputs else (lambda a: torch.as_tensor(np.asarray(a, np.float64)))
    for b, sb, u in zip(ms.blocks, scene.blocks, u0s):
        b.state = grid.init_state(conv(sb.rho0), u, conv(sb.c0), b.state.flags)
    for fb, u in zip(far, u0s[len(scene.blocks):]):
        i = ms.add_far_block(fb.origin, fb.h, fb.dims, fb.rho0, fb.u0, fb.c0, fb.flags)
        ms.blocks[i].state = grid.init_state(conv(fb.rho0), u, conv(fb.c0), ms.blocks[i].state.flags)
    for _ in range(steps):
        ms.step()
    return ms


def ms_loss_and_grad(scene, steps: int, c_target, far=()):
    """L = 1/2 sum over the reference block of (c_T - c_target)^2 and its FP64 gradients
    with respect to every block's initial velocity (reverse-mode through the whole
    Algorithm 1 schedule: steps, prior- and post-mapping, temporal alignment, and the
    far-field blocks' steps and overlap / boundary mappings)."""
    u0s = [torch.as_tensor(np.asarray(b.u0, np.float32).astype(np.float64)).clone().requires_grad_(True)
           for b in list(scene.blocks) + list(far)]
    ms = ms_forward(scene, u0s, steps, far=far)
    L = 0.5 * ((ms.blocks[0].state.c - torch.as_tensor(np.asarray(c_target), dtype=DT)) ** 2).sum()
    grads = torch.autograd.grad(L, u0s)
    return float(L.detach()), [g.detach() for g in grads], ms


def ms_loss_only(scene, u0s, steps: int, c_target, far=()):
    with torch.no_grad():
        ms = ms_forward(scene, [torch.as_tensor(np.asarray(u, np.float64)) for u in u0s], steps,
                        f32_inputs=False, far=far)
        return float(0.5 * ((ms.blocks[0].state.c - torch.as_tensor(np.asarray(c_target), dtype=DT)) ** 2).sum())
