"""Hand-written adjoint of a continuous-scale domain (reverse of the whole Algorithm 1
schedule: prior-mapping with time interpolation, sub-steps, temporal alignment,
post-mapping) against the FP64 oracle's gradient, for every block's initial velocity.

Tolerance: relative L2 <= 1e-3 per block (FP32 forward and reverse; the mapping transposes
add corner contributions atomically, in a run-dependent order)."""
import numpy as np
import pytest
import torch

import synth
from oracle import adjoint as oadj
from tests.helpers import f32
from tests.test_gpu_multiscale import gpu_multiscale

pytestmark = pytest.mark.gpu


def _case(kind):
    sc = synth.multiscale(seed=2, sphere_seed=3, scale=0.125, flow_amp=0.03, nu=0.004)
    if kind == "two_blocks":             # h = 1/1.5: two sub-steps, temporal alignment
        sc.blocks = sc.blocks[:2]
    elif kind == "integer_ratio":        # h = 1/2: two sub-steps landing on t_n + dt_0
        b1 = synth._empty_block((10, 10, 10), origin=(3.0, 4.0, 4.0), h=0.5)
        u, rho, c = synth.smooth_field(b1, 11, amp=0.03, wavelength=8.0)
        b1.u0, b1.rho0, b1.c0 = u, rho, c
        sc.blocks = [sc.blocks[0], b1]
    return sc


@pytest.mark.parametrize("kind", ["two_blocks", "integer_ratio", "three_blocks"])
def test_multiblock_adjoint_matches_fp64_oracle(lib, kind):
    from paper_1807_02284_gb300 import lbm
    sc = _case(kind)
    steps, every = 4, 2
    target = np.zeros(sc.blocks[0].shape_zyx)
    dom = gpu_multiscale(sc)
    dom.set_tape(every)
    dom.step(steps)
    c = dom.read_field(lbm.LBM_FIELD_SCALAR, lbm.LBM_F64)
    dLdc = torch.tensor(c - target.reshape(-1), dtype=torch.float32, device="cuda")
    g0 = torch.empty(3 * sc.blocks[0].flags.size, dtype=torch.float32, device="cuda")
    dom.adjoint_step(steps, dLdc, g0)
    grads = [g0]
    for i in range(1, len(sc.blocks)):
        gi = torch.empty(3 * sc.blocks[i].flags.size, dtype=torch.float32, device="cuda")
        dom.adjoint_block_grad(i, gi)
        grads.append(gi)
    dom.sync()
    dom.close()
    L, go, _ = oadj.ms_loss_and_grad(sc, steps, target)
    for i, (gg, gr) in enumerate(zip(grads, go)):
        gg = gg.cpu().numpy().astype(np.float64).reshape(sc.blocks[i].u0.shape)
        gr = gr.numpy()
        e = float(np.linalg.norm(gg - gr) / np.linalg.norm(gr))
        print(f"{kind} block {i}: |g| oracle {np.linalg.norm(gr):.3e}, rel L2 err {e:.2e}")
        assert e <= 1e-3, f"block {i}"


@pytest.mark.parametrize("refined", [False, True])
def test_farfield_adjoint_matches_fp64_oracle(lib, refined):
    """The reference block inside a far-field block (h = 1.5: aligned step, overlap and
    boundary mappings), optionally with a refined block inside the reference block: every
    block's gradient against the FP64 oracle's."""
    from paper_1807_02284_gb300 import lbm
    if refined:
        sc = _case("two_blocks")
    else:
        sc = synth.random_scene(dims=(12, 10, 10), seed=47, periodic=(False, False, False),
                                spheres=[(6.0, 5.0, 5.0, 1.6)], nu=0.01)
    fb = synth.far_block(sc.blocks[0], 1.5, 4.0, seed=6, amp=0.03)
    steps, every = 4, 2
    target = np.zeros(sc.blocks[0].shape_zyx)
    dom = gpu_multiscale(sc)
    fid = dom.add_scale_block(fb.origin, fb.h, fb.dims)
    dom.set_flags(fb.flags, block=fid)
    dom.init_macro(f32(fb.u0), rho=f32(fb.rho0), c=f32(fb.c0), block=fid)
    dom.set_tape(every)
    dom.step(steps)
    c = dom.read_field(lbm.LBM_FIELD_SCALAR, lbm.LBM_F64)
    dLdc = torch.tensor(c - target.reshape(-1), dtype=torch.float32, device="cuda")
    blocks = list(sc.blocks) + [fb]
    g0 = torch.empty(3 * blocks[0].flags.size, dtype=torch.float32, device="cuda")
    dom.adjoint_step(steps, dLdc, g0)
    grads = [g0]
    for i in range(1, len(blocks)):
        gi = torch.empty(3 * blocks[i].flags.size, dtype=torch.float32, device="cuda")
        dom.adjoint_block_grad(i, gi)
        grads.append(gi)
    dom.sync()
    dom.close()
    L, go, _ = oadj.ms_loss_and_grad(sc, steps, target, far=(fb,))
    for i, (gg, gr) in enumerate(zip(grads, go)):
        gg = gg.cpu().numpy().astype(np.float64).reshape(blocks[i].u0.shape)
        gr = gr.numpy()
        e = float(np.linalg.norm(gg - gr) / np.linalg.norm(gr))
        print(f"far field (refined {refined}) block {i}: |g| oracle {np.linalg.norm(gr):.3e}, rel L2 err {e:.2e}")
        assert e <= 1e-3, f"block {i}"
