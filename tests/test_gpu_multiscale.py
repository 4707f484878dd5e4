"""GPU parity of the continuous-scale coupling (prior-mapping, sub-cycling, temporal
alignment, post-mapping, Algorithm 1) against the FP64 oracle through the C-ABI."""
import math

import numpy as np
import pytest
import torch

import synth
from oracle import coupling, grid
from tests.helpers import f32, max_err

pytestmark = pytest.mark.gpu

U_REL = 1e-5


def gpu_multiscale(scene):
    from paper_1807_02284_gb300 import lbm
    b0 = scene.blocks[0]
    dom = lbm.Domain(b0.dims, scene.nu, periodic=scene.periodic, adaptive=scene.adaptive,
                     c_src=scene.c_src)
    for b in scene.blocks[1:]:
        dom.add_scale_block(b.origin, b.h, b.dims)
    for i, b in enumerate(scene.blocks):
        dom.set_flags(b.flags, block=i)
        dom.init_macro(f32(b.u0), rho=f32(b.rho0), c=f32(b.c0), block=i)
    return dom


def read_block(dom, i, shape):
    from paper_1807_02284_gb300 import lbm
    f = dom.read_field(lbm.LBM_FIELD_F, lbm.LBM_F64, i).reshape((27,) + shape)
    u = dom.read_field(lbm.LBM_FIELD_U, lbm.LBM_F64, i).reshape((3,) + shape)
    c = dom.read_field(lbm.LBM_FIELD_SCALAR, lbm.LBM_F64, i).reshape(shape)
    return f, u, c


def compare(dom, ms, label, f_tol=4e-7, c_tol=2e-6):
    worst = []
    for i, blk in enumerate(ms.blocks):
        shape = tuple(reversed(blk.dims))
        f, u, c = read_block(dom, i, shape)
        uo = blk.state.u.numpy()
        umax = float(np.abs(uo).max())
        eu, ef, ec = max_err(u, uo), max_err(f, blk.state.f.numpy()), max_err(c, blk.state.c.numpy())
        worst.append((i, eu, ef, ec, umax))
        print(f"{label} block {i}: |du|={eu:.2e} (max|u| {umax:.3f}) |df|={ef:.2e} |dc|={ec:.2e}")
    for i, eu, ef, ec, umax in worst:
        assert eu <= U_REL * max(umax, 1e-3), f"{label} block {i} velocity"
        assert ef <= f_tol, f"{label} block {i} populations"
        assert ec <= c_tol, f"{label} block {i} scalar"


def test_block_info_reports_scales(lib):
    sc = synth.multiscale(scale=0.25)
    dom = gpu_multiscale(sc)
    i1, i2 = dom.info(1), dom.info(2)
    assert (i1.substeps, i2.substeps) == (2, 3)
    assert i1.nu == pytest.approx(sc.nu * 1.5) and i2.nu == pytest.approx(sc.nu * 2.25)
    flags = dom.read_field(4, 2, block=2).reshape(tuple(reversed(sc.blocks[2].dims)))
    assert (flags[0] & synth.GHOST).all() and not (flags[1:-1, 1:-1, 1:-1] & synth.GHOST).any()
    dom.close()


@pytest.mark.parametrize("steps", [1, 4])
def test_three_block_parity_non_integer_ratios(lib, steps):
    """Reduced copy (1/4 of every length) of the 3-block scene: s0 32^3, s1 24^3 at h=1/1.5,
    s2 16^3 at h=1/2.25, 8 spheres, inflow with noise, and a seeded smooth flow, density
    and scalar field sampled by every block so that every mapping moves non-trivial data."""
    sc = synth.multiscale(scale=0.25, nu=2e-3, flow_amp=0.06)
    dom = gpu_multiscale(sc)
    ms = coupling.MultiScale.build(sc)
    for _ in range(steps):
        dom.step(1)
        ms.step()
    dom.sync()
    compare(dom, ms, f"3-block x{steps}")
    dom.close()


def test_graph_replay_matches_direct_steps_multiblock(lib):
    """lbm_step(n) replays captured graphs of the concurrent fork/join schedule; it must give
    the same bits as n single steps launched directly."""
    from paper_1807_02284_gb300 import lbm
    sc = synth.multiscale(scale=0.25, nu=2e-3, flow_amp=0.06)
    a = gpu_multiscale(sc)
    b = gpu_multiscale(sc)
    a.step(40)
    for _ in range(40):
        b.step(1)
    for i in range(3):
        fa = a.read_field(lbm.LBM_FIELD_F, lbm.LBM_F32, i)
        fb = b.read_field(lbm.LBM_FIELD_F, lbm.LBM_F32, i)
        assert np.array_equal(fa, fb), f"block {i}"
        assert np.array_equal(a.read_field(lbm.LBM_FIELD_SCALAR, lbm.LBM_F32, i),
                              b.read_field(lbm.LBM_FIELD_SCALAR, lbm.LBM_F32, i))
    a.close()
    b.close()


def test_integer_ratio_two_block_parity(lib):
    """alpha = 2 two-block case on a periodic Taylor-Green field (no temporal interpolation:
    two sub-steps land exactly on t_n + dt_0)."""
    sc = synth.taylor_green(24, nz=12, re=60)
    b1 = synth._empty_block((16, 14, 10), origin=(5.0, 4.5, 3.0), h=0.5)
    k = 2 * math.pi / 24
    xs, ys, zs = b1.node_coords()
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    b1.u0[0] = 0.05 * np.sin(k * X) * np.cos(k * Y)
    b1.u0[1] = -0.05 * np.cos(k * X) * np.sin(k * Y)
    b1.c0[:] = np.exp(-((X - 9) ** 2 + (Y - 8) ** 2) / 8.0)
    sc.blocks.append(b1)
    dom = gpu_multiscale(sc)
    ms = coupling.MultiScale.build(sc)
    for _ in range(3):
        dom.step(1)
        ms.step()
    compare(dom, ms, "alpha=2")
    dom.close()


def test_uniform_flow_stays_uniform_full_size(lib):
    """Full-size 3-block geometry (128^3, 96^3 at h=1/1.5, 64^3 at h=1/2.25), periodic s0, no
    obstacles, uniform flow: every step, mapping and interpolation keeps it uniform."""
    from paper_1807_02284_gb300 import lbm
    full = synth.multiscale(scale=1.0)
    blocks = []
    for b in full.blocks:
        nb = synth._empty_block(b.dims, origin=b.origin, h=b.h)
        nb.u0[0], nb.u0[1], nb.u0[2] = 0.05, -0.02, 0.01
        blocks.append(nb)
    sc = synth.Scene(blocks=blocks, periodic=(True, True, True), nu=1e-5)
    dom = gpu_multiscale(sc)
    dom.step(3)
    dom.sync()
    for i, b in enumerate(blocks):
        u = dom.read_field(lbm.LBM_FIELD_U, lbm.LBM_F32, i).reshape(3, -1)
        err = np.abs(u - np.array([[0.05], [-0.02], [0.01]], np.float32)).max()
        print(f"uniform full-size block {i}: max |u - u0| = {err:.2e}")
        assert err < 2e-6
    dom.close()


def test_full_size_reference_block_far_field_sampled(lib):
    """Full-size 3-block scene: one reference step at s0 nodes away from the refined blocks
    is the single-block update of the GPU's own t_n state, checked node by node."""
    from paper_1807_02284_gb300 import lbm
    sc = synth.multiscale(scale=1.0)
    dom = gpu_multiscale(sc)
    dom.step(3)
    b0 = sc.blocks[0]
    shape = b0.shape_zyx
    f = dom.read_field(lbm.LBM_FIELD_F, lbm.LBM_F32, 0).reshape((27,) + shape)
    u = dom.read_field(lbm.LBM_FIELD_U, lbm.LBM_F32, 0).reshape((3,) + shape)
    c = dom.read_field(lbm.LBM_FIELD_SCALAR, lbm.LBM_F32, 0).reshape(shape)
    dom.step(1)
    f1 = dom.read_field(lbm.LBM_FIELD_F, lbm.LBM_F32, 0).reshape((27,) + shape)
    st = grid.State(torch.from_numpy(f.astype(np.float64)), torch.from_numpy(u.astype(np.float64)),
                    torch.from_numpy(c.astype(np.float64)), torch.from_numpy(b0.flags.copy()))
    rng = np.random.default_rng(1)
    s1 = sc.blocks[1]
    lo = np.array(s1.origin) - 2
    hi = np.array(s1.origin) + (np.array(s1.dims) - 1) * s1.h + 2
    pts = []
    while len(pts) < 3000:
        p = rng.integers(0, 128, 3)   # (x, y, z)
        if np.all(p >= lo) and np.all(p <= hi):
            continue
        pts.append(p)
    pts = np.array(pts)
    x, y, z = (torch.from_numpy(pts[:, i].astype(np.int64)) for i in range(3))
    fo, uo, co = grid.step_cells(st, grid.Params(nu=sc.nu, periodic=sc.periodic, c_src=sc.c_src),
                                 z, y, x)
    got = f1[:, pts[:, 2], pts[:, 1], pts[:, 0]].T
    err = np.abs(got - fo.numpy()).max()
    print(f"far-field sampled s0: |df| = {err:.2e}")
    assert err < 2e-7
    dom.close()


def test_scale_block_argument_checks(lib):
    from paper_1807_02284_gb300 import lbm
    dom = lbm.Domain((16, 16, 16), 1e-3)
    with pytest.raises(lbm.LBMError) as ei:               # far field not around s0
        dom.add_scale_block((2, 2, 2), 1.5, (8, 8, 8))
    assert ei.value.status == lbm.LBM_ERR_INVALID_ARG
    with pytest.raises(lbm.LBMError) as ei:
        dom.add_scale_block((10, 10, 10), 0.5, (20, 8, 8))          # sticks out of s0
    assert ei.value.status == lbm.LBM_ERR_INVALID_ARG
    with pytest.raises(lbm.LBMError):
        dom.add_scale_block((2, 2, 2), 0.5, (3, 8, 8))              # too thin
    dom.add_scale_block((2, 2, 2), 0.5, (8, 8, 8))
    with pytest.raises(lbm.LBMError):
        dom.add_scale_block((2, 2, 2), 0.75, (8, 8, 8))             # not coarse to fine
    dom.close()
    d16 = lbm.Domain((16, 16, 16), 1e-3, storage="fp16")
    with pytest.raises(lbm.LBMError) as ei:
        d16.add_scale_block((2, 2, 2), 0.5, (8, 8, 8))
    assert ei.value.status == lbm.LBM_ERR_UNSUPPORTED
    d16.close()


@pytest.mark.parametrize("kind", ["nested", "far"])
def test_schedule_exact_on_affine_scalar_transport(lib, kind):
    """The exact Algorithm 1 case of the oracle pin (uniform flow, scalar affine in space,
    blocks at h = 1/1.5 and 1/2.25, or a refined block inside s0 inside a far block at h = 2):
    every checked node of every block holds c0 + G . (x - U n) after each reference step, to
    float32 rounding, and agrees with the oracle."""
    from paper_1807_02284_gb300 import lbm
    from tests import test_oracle_schedule as ts
    if kind == "nested":
        sc, far = ts.nested_scene(), None
    else:
        sc, far = ts.far_scene()
    dom = gpu_multiscale(sc)
    blocks = list(sc.blocks)
    if far is not None:
        fid = dom.add_scale_block(far.origin, far.h, far.dims)
        dom.set_flags(far.flags, block=fid)
        dom.init_macro(f32(far.u0), rho=f32(far.rho0), c=f32(far.c0), block=fid)
        blocks.append(far)
    ms = ts.build(kind)
    for n in range(1, 4):
        dom.step(1)
        ms.step()
        for i, (b, m) in enumerate(zip(blocks, ts.checked_masks(ms, n))):
            c = dom.read_field(lbm.LBM_FIELD_SCALAR, lbm.LBM_F64, i).reshape(b.shape_zyx)
            want = ts.exact_scalar(b.origin, b.h, b.dims, n)
            e_exact = float(np.abs(c - want)[m].max())
            e_oracle = max_err(c, ms.blocks[i].state.c.numpy())
            print(f"{kind} step {n} block {i}: |c - exact| = {e_exact:.2e}, "
                  f"|c - oracle| = {e_oracle:.2e}")
            assert e_exact < 3e-6 and e_oracle < 3e-6, (n, i)
    dom.close()


def _oracle_blocks_from_gpu(dom, sc):
    """Oracle blocks holding the GPU's current float32 states (widened exactly) and flags."""
    from paper_1807_02284_gb300 import lbm
    out = []
    for i, b in enumerate(sc.blocks):
        f, u, c = read_block(dom, i, b.shape_zyx)
        fl = dom.read_field(lbm.LBM_FIELD_FLAGS, lbm.LBM_U8, i).reshape(b.shape_zyx) & 0x0F
        st = grid.State(torch.from_numpy(f), torch.from_numpy(u), torch.from_numpy(c),
                        torch.from_numpy(fl.astype(np.uint8)))
        out.append(coupling.Blk(origin=np.array(b.origin, dtype=np.float64), h=float(b.h),
                                dims=tuple(b.dims), state=st,
                                params=grid.Params(nu=sc.nu / b.h, periodic=(False,) * 3)))
    return out


def _check_mapped(label, src, dst, z, y, x, rng, n=3000, f_tol=4e-7, c_tol=2e-6):
    """dst's stored values at sampled nodes (z, y, x) against the oracle's trilinear
    interpolation of src's state at their positions followed by the K_hat mapping
    (Sec. 3.2, Sec. 4.2.2); nodes whose corners are all obstacles hold the rest state."""
    from oracle import cmr
    assert z.numel() > 0, label
    pick = torch.from_numpy(rng.choice(z.numel(), size=min(n, z.numel()), replace=False))
    z, y, x = z[pick], y[pick], x[pick]
    f, c, ok = coupling.interpolate(src, src.state.f, src.state.c,
                                    coupling.node_positions(dst, z, y, x))
    fm = coupling.map_populations(f[ok], coupling.k_hat(src, dst))
    _, um = cmr.macros(fm)
    got_f = dst.state.f[:, z, y, x].T
    got_u = dst.state.u[:, z, y, x].T
    got_c = dst.state.c[z, y, x]
    ef = float((got_f[ok] - fm).abs().max())
    eu = float((got_u[ok] - um).abs().max())
    ec = float((got_c[ok] - c[ok]).abs().max())
    umax = float(um.abs().max())
    print(f"{label}: {int(pick.numel())} nodes ({int((~ok).sum())} at rest) |df|={ef:.2e} "
          f"|du|={eu:.2e} (max|u| {umax:.3f}) |dc|={ec:.2e}")
    assert ef <= f_tol and eu <= U_REL * max(umax, 1e-3) and ec <= c_tol, label
    if bool((~ok).any()):
        rest = cmr.equilibrium(torch.ones(1, dtype=torch.float64),
                               torch.zeros(1, 3, dtype=torch.float64))[0]
        assert float((got_f[~ok] - rest).abs().max()) <= f_tol, label


def _span_nodes(tgt, src):
    """Nodes of tgt inside src's interior span (Sec. 4.2.5 post-mapping targets) that are
    neither ghost nor obstacle nodes of tgt."""
    lo, hi = src.interior_lo_hi()
    zz, yy, xx = torch.meshgrid(*(torch.arange(n) for n in reversed(tgt.dims)), indexing="ij")
    zz, yy, xx = zz.reshape(-1), yy.reshape(-1), xx.reshape(-1)
    pos = coupling.node_positions(tgt, zz, yy, xx)
    inside = torch.ones(pos.shape[0], dtype=torch.bool)
    for a in range(3):
        inside &= (pos[:, a] >= lo[a] - 1e-9) & (pos[:, a] <= hi[a] + 1e-9)
    inside &= (tgt.state.flags[zz, yy, xx] & (coupling.GHOST | coupling.SOLID)) == 0
    sel = torch.nonzero(inside).flatten()
    return zz[sel], yy[sel], xx[sel]


def _drop_touching(src, dst, nodes, finer):
    """Leave out dst nodes whose trilinear source cell in src has a corner of non-zero weight
    among src's nodes inside the finer block's interior span: those corners are post-mapped
    from the finer block after dst's mapping was taken within the step."""
    z, y, x = nodes
    lo, hi = finer.interior_lo_hi()
    a_lo = np.ceil((lo - src.origin) / src.h - 1e-9)
    a_hi = np.floor((hi - src.origin) / src.h + 1e-9)
    q = (coupling.node_positions(dst, z, y, x) - torch.as_tensor(src.origin)) / src.h
    touch = torch.ones(z.shape, dtype=torch.bool)
    for a in range(3):
        i0 = torch.floor(q[:, a] + 1e-9).long()
        i1 = torch.where(q[:, a] - i0.to(q.dtype) > 1e-9, i0 + 1, i0)   # weight-0 corner ignored
        touch &= (i1 >= int(a_lo[a])) & (i0 <= int(a_hi[a]))
    keep = ~touch
    return z[keep], y[keep], x[keep]


def test_full_size_mappings_sampled(lib):
    """Full-size 3-block scene with a seeded non-uniform flow and the 8 obstacles, after two
    reference steps: sampled nodes of every mapping of Algorithm 1 against the oracle's
    interpolation and K_hat mapping of the GPU's own source state -- the ghost layers of s1
    (from s0) and s2 (from s1), and the post-mapped nodes of s0 from s1 (about 240k entries:
    the large-mapping kernel variant), of s0 from s2 and of s1 from s2.  Within one step s1
    is post-mapped into s0 before s2 is post-mapped into s1, so s0 targets whose s1 cell
    touches s1's nodes inside s2's span are left out of the s1 -> s0 check."""
    sc = synth.multiscale(scale=1.0, flow_amp=0.06)
    dom = gpu_multiscale(sc)
    dom.step(2)
    dom.sync()
    s0, s1, s2 = _oracle_blocks_from_gpu(dom, sc)
    rng = np.random.default_rng(12)
    for label, src, dst in (("s1 ghost layer from s0", s0, s1), ("s2 ghost layer from s1", s1, s2)):
        g = ((dst.state.flags & coupling.GHOST) != 0) & ((dst.state.flags & coupling.SOLID) == 0)
        nodes = torch.nonzero(g, as_tuple=True)
        if src is s1:
            nodes = _drop_touching(s1, s2, nodes, s2)
        _check_mapped(label, src, dst, *nodes, rng)
    nodes = _span_nodes(s0, s1)
    assert nodes[0].numel() >= 155_000                    # the large-mapping variant
    _check_mapped("s0 post-mapped from s1", s1, s0, *_drop_touching(s1, s0, nodes, s2), rng)
    z, y, x = _span_nodes(s0, s2)
    _check_mapped("s0 post-mapped from s2", s2, s0, z, y, x, rng)
    z, y, x = _span_nodes(s1, s2)
    _check_mapped("s1 post-mapped from s2", s2, s1, z, y, x, rng)
    dom.close()


@pytest.mark.parametrize("steps", [1, 3])
def test_obstacle_walls_on_refined_blocks(lib, steps):
    """The second-order wall on the obstacles' surfaces (Sec. 6.1, reading of the regularized
    on-node wall) in every block of the reduced 3-block scene, whose 8 spheres sit inside the
    refined blocks: parity with the oracle evaluating the same wall on each block, the
    mappings treating every obstacle voxel as an obstacle."""
    sc = synth.multiscale(scale=0.25, nu=2e-3, flow_amp=0.06)
    dom = gpu_multiscale(sc)
    dom.set_walls((False,) * 6, obstacles=True)
    for i, b in enumerate(sc.blocks):          # re-initialise: surface voxels start at rest
        dom.init_macro(f32(b.u0), rho=f32(b.rho0), c=f32(b.c0), block=i)
    ms = coupling.MultiScale.build(sc, obstacle_walls=True)
    surf = 0
    for i, b in enumerate(ms.blocks):
        s = grid.surface_voxels(b.state.flags, b.params.periodic)
        surf += int(s.sum())
        fl = dom.read_field(4, 2, block=i).reshape(b.state.flags.shape)
        assert np.array_equal((fl & 64) != 0, s.numpy()), f"block {i} surface voxels"
    assert surf > 0
    for _ in range(steps):
        dom.step(1)
        ms.step()
    dom.sync()
    compare(dom, ms, f"obstacle walls x{steps}")
    dom.close()
