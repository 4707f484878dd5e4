"""torch.autograd wrapper of the hand-written adjoint (lbm_set_tape / lbm_adjoint_step).

``SmokeRollout.apply(u0, dom, steps, every, rho0, c0)`` initialises block 0 of ``dom`` (an
``lbm.Domain`` in any configuration the adjoint covers: periodic or open faces, walls,
obstacles, inflow nodes, FP32 or FP16-shifted storage) at the equilibrium of (rho0, u0, c0),
advances it ``steps`` steps with a checkpoint every ``every`` steps, and returns block 0's
final scalar field (float32, one value per node, index (z*ny + y)*nx + x).  Its backward
runs the library's reverse sweep and returns dL/du0 with the layout of u0 (3 planes).  Only
argument marshalling happens here.
"""
from __future__ import annotations

import torch

from . import lbm


class SmokeRollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, dom, steps, every, rho0=None, c0=None):
        if not u0.is_cuda or u0.dtype != torch.float32:
            raise ValueError("u0 must be a float32 CUDA tensor")
        u = u0.detach().contiguous()
        dom.init_macro(u, rho=None if rho0 is None else rho0.detach().float().contiguous(),
                       c=None if c0 is None else c0.detach().float().contiguous())
        dom.set_tape(int(every))
        dom.step(int(steps))
        n = dom.n_nodes()
        c = torch.empty(n, dtype=torch.float32, device=u0.device)
        dom.read_field(lbm.LBM_FIELD_SCALAR, lbm.LBM_F32, out=c)
        ctx.dom = dom
        ctx.steps = int(steps)
        ctx.shape = u0.shape
        return c

    @staticmethod
    def backward(ctx, grad_c):
        n = ctx.dom.n_nodes()
        g = torch.empty(3 * n, dtype=torch.float32, device=grad_c.device)
        ctx.dom.adjoint_step(ctx.steps, grad_c.detach().float().contiguous(), g)
        ctx.dom.sync()
        return g.view(ctx.shape), None, None, None, None, None


def smoke_rollout(u0, dom, steps, every, rho0=None, c0=None):
    return SmokeRollout.apply(u0, dom, steps, every, rho0, c0)
