"""Shared helpers of the GPU parity tests: run a seeded ``synth`` scene through the C-ABI
library and through the FP64 oracle on identical (float32-rounded) inputs."""
import numpy as np
import torch

import synth
from oracle import grid


def f32(a):
    """Inputs are handed to the library as float32; the oracle gets the same rounded values."""
    return np.asarray(a, dtype=np.float32)


def gpu_domain(scene, storage="fp32", block=0, grad_mode="lagged"):
    from paper_1807_02284_gb300 import lbm
    b = scene.blocks[block]
    dom = lbm.Domain(b.dims, scene.nu, periodic=scene.periodic, storage=storage,
                     adaptive=scene.adaptive, c_src=scene.c_src, grad_mode=grad_mode)
    dom.set_flags(b.flags)
    dom.init_macro(f32(b.u0), rho=f32(b.rho0), c=f32(b.c0))
    return dom


def gpu_state(dom, shape_zyx, block=0, dtype=None):
    """(f, u, c) of a block as float64 numpy arrays shaped [27|3][z][y][x]."""
    from paper_1807_02284_gb300 import lbm
    dt = lbm.LBM_F64 if dtype is None else dtype
    f = dom.read_field(lbm.LBM_FIELD_F, dt, block).reshape((27,) + tuple(shape_zyx))
    u = dom.read_field(lbm.LBM_FIELD_U, dt, block).reshape((3,) + tuple(shape_zyx))
    c = dom.read_field(lbm.LBM_FIELD_SCALAR, dt, block).reshape(tuple(shape_zyx))
    return f.astype(np.float64), u.astype(np.float64), c.astype(np.float64)


def oracle_state(scene, block=0):
    b = scene.blocks[block]
    return grid.init_state(f32(b.rho0).astype(np.float64), f32(b.u0).astype(np.float64),
                           f32(b.c0).astype(np.float64), b.flags)


def oracle_params(scene, grad_mode="lagged"):
    return grid.Params(nu=scene.nu, periodic=scene.periodic, adaptive=scene.adaptive,
                       c_src=scene.c_src, grad_mode=grad_mode)


def state_from_arrays(f, u, c, flags):
    return grid.State(torch.as_tensor(f), torch.as_tensor(u), torch.as_tensor(c),
                      torch.as_tensor(np.asarray(flags).astype(np.uint8)))


def max_err(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max())
