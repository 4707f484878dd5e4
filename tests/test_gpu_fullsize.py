"""Full-size checks: the 256^3 smoke plume (inflow disk, voxelised sphere, open faces) in the
launch configuration the benchmark times, compared with the oracle on sampled nodes, and
the FP16 equilibrium-shifted storage compared with the FP32 path and the oracle."""
import numpy as np
import pytest
import torch

import synth
from oracle import grid
from tests.helpers import f32, gpu_domain, gpu_state, max_err, oracle_params, oracle_state

pytestmark = pytest.mark.gpu


def _sample_nodes(b, rng, n_random=3000, n_near=600, n_face=600):
    nz, ny, nx = b.shape_zyx
    pick = [np.stack([rng.integers(0, nz, n_random), rng.integers(0, ny, n_random),
                      rng.integers(0, nx, n_random)], 1)]
    fl = b.flags
    inflow = np.argwhere((fl & synth.INFLOW) != 0)
    pick.append(inflow)
    solid = (fl & synth.SOLID) != 0
    near = np.zeros_like(solid)
    for ax in range(3):
        for s in (-1, 1):
            near |= np.roll(solid, s, axis=ax)
    near &= ~solid
    cand = np.argwhere(near)
    pick.append(cand[rng.choice(len(cand), min(n_near, len(cand)), replace=False)])
    zf = rng.integers(0, nz, n_face)
    yf = rng.integers(0, ny, n_face)
    xf = rng.choice([0, nx - 1], n_face)
    pick.append(np.stack([zf, yf, xf], 1))
    return np.unique(np.concatenate(pick), axis=0)


def test_plume_256_sampled_parity(lib):
    """Advance the full 256^3 plume 24 steps on the GPU (captured-graph path), then check
    one more step node by node against the oracle evaluated from the GPU's step-24 state."""
    from paper_1807_02284_gb300 import lbm
    sc = synth.plume(256)
    b = sc.blocks[0]
    dom = gpu_domain(sc)
    dom.step(24)
    dom.sync()
    f, u, c = gpu_state(dom, b.shape_zyx, dtype=lbm.LBM_F32)
    dom.step(1)
    f1, u1, c1 = gpu_state(dom, b.shape_zyx, dtype=lbm.LBM_F32)
    st = grid.State(torch.from_numpy(f), torch.from_numpy(u), torch.from_numpy(c),
                    torch.from_numpy(b.flags.copy()))
    del f, u, c
    nodes = _sample_nodes(b, np.random.default_rng(0))
    z, y, x = (torch.from_numpy(nodes[:, i].astype(np.int64)) for i in range(3))
    fo, uo, co = grid.step_cells(st, oracle_params(sc), z, y, x)
    zi, yi, xi = nodes[:, 0], nodes[:, 1], nodes[:, 2]
    eu = np.abs(u1[:, zi, yi, xi].T - uo.numpy()).max()
    ef = np.abs(f1[:, zi, yi, xi].T - fo.numpy()).max()
    ec = np.abs(c1[zi, yi, xi] - co.numpy()).max()
    umax = float(np.abs(uo.numpy()).max())
    print(f"plume 256 sampled ({len(nodes)} nodes): |du|={eu:.2e} |df|={ef:.2e} |dc|={ec:.2e}")
    assert eu <= 1e-5 * umax
    assert ef <= 2e-7
    assert ec <= 1e-6
    dom.close()


def test_fp16_shifted_storage_against_fp32_and_oracle(lib):
    """FP16 equilibrium-shifted storage: error against the FP32 GPU path and the FP64
    oracle on a plume-shaped scene after 20 steps (binary16 keeps 11 significant bits of
    f_i - w_i; the bound below is 2e-3 of max|u|)."""
    sc = synth.random_scene(dims=(48, 40, 40), seed=21, periodic=(False, False, False),
                            spheres=[(20.0, 20.0, 20.0, 6.0)], inflow=(20, 20, 8.0, 0.1),
                            nu=1e-4)
    b = sc.blocks[0]
    d32 = gpu_domain(sc, "fp32")
    d16 = gpu_domain(sc, "fp16")
    st = oracle_state(sc)
    p = oracle_params(sc)
    for _ in range(20):
        d32.step(1)
        d16.step(1)
        st = grid.step(st, p)
    _, u32, c32 = gpu_state(d32, b.shape_zyx)
    _, u16, c16 = gpu_state(d16, b.shape_zyx)
    uo = st.u.numpy()
    umax = float(np.abs(uo).max())
    e16_32 = max_err(u16, u32)
    e16_or = max_err(u16, uo)
    e32_or = max_err(u32, uo)
    r32 = d32.reduce()
    r16 = d16.reduce()
    print(f"fp16 vs fp32 |du|={e16_32:.2e}, fp16 vs oracle {e16_or:.2e}, fp32 vs oracle "
          f"{e32_or:.2e}, max|u|={umax:.3f}, mass fp16/fp32-1 = {r16[0] / r32[0] - 1:.2e}")
    assert e32_or <= 1e-5 * umax
    assert e16_or <= 2e-3 * umax
    assert abs(r16[0] / r32[0] - 1) < 1e-4
    d32.close()
    d16.close()


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_largest_sizes_take_the_64_bit_index_path_exactly(lib, storage):
    """A block with 27 N >= 2^32 (here 544^3, 161 M nodes, a 35 GB FP32 state) runs the 64-bit
    index instance of the collide-stream kernel.  Its result is checked through a property
    that holds at any size: a periodic 544^3 domain tiled 17 x 17 x 17 from a 32^3 seeded
    scene (sphere, random velocity, density and scalar) must hold, after 3 steps, exactly the
    tiled state of the 32^3 domain, which runs the 32-bit instance (same per-node arithmetic,
    other index arithmetic)."""
    from paper_1807_02284_gb300 import lbm
    rep = 17
    sc = synth.random_scene(dims=(32, 32, 32), seed=61, periodic=(True, True, True),
                            spheres=[(16.0, 15.0, 17.0, 5.0)], nu=1e-3)
    b = sc.blocks[0]
    small = gpu_domain(sc, storage)
    big_dims = tuple(d * rep for d in b.dims)
    assert 27 * int(np.prod(big_dims)) >= 2 ** 32
    big = lbm.Domain(big_dims, sc.nu, periodic=sc.periodic, storage=storage,
                     adaptive=sc.adaptive, c_src=sc.c_src)
    big.set_flags(np.tile(b.flags, (rep, rep, rep)))
    dev = torch.device("cuda")
    u = torch.tensor(f32(b.u0), device=dev).repeat(1, rep, rep, rep).contiguous()
    rho = torch.tensor(f32(b.rho0), device=dev).repeat(rep, rep, rep).contiguous()
    c = torch.tensor(f32(b.c0), device=dev).repeat(rep, rep, rep).contiguous()
    big.init_macro(u, rho=rho, c=c)
    del u, rho, c
    small.step(3)
    big.step(3)
    N = int(np.prod(big_dims))
    for field, comps in ((lbm.LBM_FIELD_U, 3), (lbm.LBM_FIELD_SCALAR, 1), (lbm.LBM_FIELD_RHO, 1)):
        s = torch.tensor(small.read_field(field, lbm.LBM_F32), device=dev)
        s = s.reshape((comps,) + b.shape_zyx).repeat(1, rep, rep, rep)
        g = torch.empty(comps * N, dtype=torch.float32, device=dev)
        big.read_field(field, lbm.LBM_F32, out=g)
        big.sync()
        assert torch.equal(g.reshape(s.shape), s), field
        del g, s
    small.close()
    big.close()
