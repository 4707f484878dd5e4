"""GPU parity of dynamic scale construction (Sec. 5) against the FP64 oracle through the
C-ABI: detection count and box (integers, exact), placement of the new block (exact), the
started block's state, and the multi-block steps after building and after rebuilding."""
import numpy as np
import pytest

import synth
from oracle import coupling, dynamic
from tests.test_gpu_multiscale import compare, gpu_multiscale

pytestmark = pytest.mark.gpu

MASK = 1 | 4 | 8          # obstacle, scalar source, ghost bits (near-obstacle is derived)


def _scene():
    return synth.random_scene(dims=(30, 26, 20), seed=31, periodic=(False, False, False),
                              spheres=[(17.0, 13.0, 10.0, 3.5)], inflow=(13, 10, 4.0, 0.09),
                              nu=0.004)


def _thresholds(ms, q_g=0.97, q_u=0.8, gap=2e-6):
    """Thresholds at quantiles of the oracle's fields, moved off any sample by `gap` so that
    the GPU (FP32) and the oracle (FP64) take the same decision at every node."""
    b = ms.blocks[0]
    _, _, g, um = dynamic.detect(b.state, b.params.periodic, 0.0, 0.0)
    g, um = g.numpy().ravel(), um.numpy().ravel()

    def clear(v, t):
        while np.abs(v - t).min() < gap:
            t += 3 * gap
        return t
    return clear(g, float(np.quantile(g, q_g))), clear(um, float(np.quantile(um, q_u)))


def test_detection_count_and_box_match_oracle(lib):
    sc = _scene()
    dom = gpu_multiscale(sc)
    ms = coupling.MultiScale.build(sc)
    for _ in range(5):
        dom.step(1)
        ms.step()
    g_thr, u_thr = _thresholds(ms)
    n_o, box_o, _, _ = dynamic.detect(ms.blocks[0].state, sc.periodic, g_thr, u_thr)
    n_g, box_g = dom.detect_region(g_thr, u_thr)
    print("detect", n_g, box_g, n_o, box_o)
    assert n_o > 0 and n_g == n_o and box_g == box_o
    dims = sc.blocks[0].dims                        # a localised region, not the whole block
    assert any(box_o[3 + a] - box_o[a] + 1 < dims[a] for a in range(3))
    assert dom.detect_region(1e9, 0.0) == (0, None)
    dom.close()


def test_started_block_and_following_steps_match_oracle(lib):
    from paper_1807_02284_gb300 import lbm
    sc = _scene()
    dom = gpu_multiscale(sc)
    ms = coupling.MultiScale.build(sc)
    for _ in range(3):
        dom.step(1)
        ms.step()
    origin, h, dims = (5.25, 4.5, 3.75), 1 / 1.5, (30, 27, 19)   # covers the sphere
    bid = dom.add_scale_block(origin, h, dims)
    dom.init_block_from_parent(bid)
    i = dynamic.add_block_from_parent(ms, origin, h, dims)
    assert bid == i == 1
    fl = dom.read_field(lbm.LBM_FIELD_FLAGS, lbm.LBM_U8, 1).reshape(tuple(reversed(dims)))
    assert np.array_equal(fl & MASK, ms.blocks[1].state.flags.numpy() & MASK)
    assert (fl & 1).any()                       # the sphere reaches into the new block
    compare(dom, ms, "started")
    for _ in range(3):
        dom.step(1)
        ms.step()
    compare(dom, ms, "stepped")
    dom.close()


def test_build_and_rebuild_dynamic_scale_match_oracle(lib):
    sc = _scene()
    dom = gpu_multiscale(sc)
    ms = coupling.MultiScale.build(sc)
    for _ in range(4):
        dom.step(1)
        ms.step()
    h, margin = 1 / 1.5, 2
    ref = sc.blocks[0].dims
    for rebuild in (False, True):
        g_thr, u_thr = _thresholds(ms, q_g=0.99, q_u=0.6)
        bid = dom.build_dynamic_scale(h, g_thr, u_thr, margin=margin, replace_last=rebuild)
        if rebuild:
            dynamic.remove_last_block(ms)
        n, box, _, _ = dynamic.detect(ms.blocks[0].state, sc.periodic, g_thr, u_thr)
        assert n > 0 and bid == 1
        o, d = dynamic.place(box, (0.0, 0.0, 0.0), 1.0, h, margin, ref)
        dynamic.add_block_from_parent(ms, o, h, d)
        info = dom.info(1)
        print("dynamic block", tuple(info.dims), tuple(info.origin), "oracle", d, o)
        assert tuple(info.dims) == d
        assert np.allclose(tuple(info.origin), o, atol=1e-12)
        compare(dom, ms, f"built (rebuild={rebuild})")
        for _ in range(3):
            dom.step(1)
            ms.step()
        compare(dom, ms, f"after build (rebuild={rebuild})")
    dom.close()


def test_dynamic_scale_argument_checks(lib):
    from paper_1807_02284_gb300 import lbm
    sc = _scene()
    dom = gpu_multiscale(sc)
    with pytest.raises(lbm.LBMError) as ei:
        dom.build_dynamic_scale(0.5, 0.0, 0.0, replace_last=True)   # no refined block yet
    assert ei.value.status == lbm.LBM_ERR_INVALID_ARG
    with pytest.raises(lbm.LBMError) as ei:
        dom.build_dynamic_scale(1.0, 0.0, 0.0)                      # not finer than s0
    assert ei.value.status == lbm.LBM_ERR_INVALID_ARG
    assert dom.build_dynamic_scale(0.5, 1e9, 0.0) == -1             # nothing selected
    a = dom.add_scale_block((2.0, 2.0, 2.0), 0.5, (10, 10, 10))
    b = dom.add_scale_block((3.0, 3.0, 3.0), 0.5, (8, 8, 8))
    with pytest.raises(lbm.LBMError) as ei:
        dom.remove_scale_block(a)                                   # not the last block
    assert ei.value.status == lbm.LBM_ERR_INVALID_ARG
    with pytest.raises(lbm.LBMError):
        dom.remove_scale_block(0)
    with pytest.raises(lbm.LBMError):
        dom.init_block_from_parent(0)
    dom.remove_scale_block(b)
    dom.remove_scale_block(a)
    dom.step(2)
    dom.sync()
    dom.close()


def test_static_scales_match_oracle(lib):
    """Static construction (Sec. 5): 3 scales (h = 1, 0.75, 0.5) around the sphere with a
    wake along x; the placed blocks equal the oracle's, their started states and the
    following steps match."""
    sc = _scene()
    dom = gpu_multiscale(sc)
    ms = coupling.MultiScale.build(sc)
    for _ in range(2):
        dom.step(1)
        ms.step()
    n = dom.build_static_scales(3, 0.5, 4.0, wake=6.0, flow_axis=0)
    plan = dynamic.static_scales(sc.blocks[0].flags, 3, 0.5, 4.0, 6.0, flow_axis=0)
    assert n == len(plan) == 2
    for i, (o, h, d) in enumerate(plan, start=1):
        info = dom.info(i)
        assert tuple(info.dims) == d and abs(info.h - h) < 1e-12
        assert np.allclose(tuple(info.origin), o, atol=1e-12)
        dynamic.add_block_from_parent(ms, o, h, d)
    compare(dom, ms, "static scales started")
    for _ in range(2):
        dom.step(1)
        ms.step()
    compare(dom, ms, "static scales stepped")
    dom.close()


def test_shadow_scales_match_oracle(lib):
    """Static construction with the soft-shadow wake (Sec. 5): the inflow disk lights the
    sphere, 4 scales (h = 1, 5/6, 2/3, 1/2); the blocks placed from the GPU's integer
    visibility counts equal the oracle's (which differ from the straight wake's here), their
    started states and the following steps match."""
    sc = _scene()
    dom = gpu_multiscale(sc)
    ms = coupling.MultiScale.build(sc)
    for _ in range(2):
        dom.step(1)
        ms.step()
    n = dom.build_static_scales_shadow(4, 0.5, 2.0, wake=6.0, flow_axis=0, n_light=16)
    plan = dynamic.shadow_scales(sc.blocks[0].flags, 4, 0.5, 2.0, 6.0, flow_axis=0, n_light=16)
    assert plan != dynamic.static_scales(sc.blocks[0].flags, 4, 0.5, 2.0, 6.0, flow_axis=0)
    assert n == len(plan) == 3
    for i, (o, h, d) in enumerate(plan, start=1):
        info = dom.info(i)
        assert tuple(info.dims) == d and abs(info.h - h) < 1e-12
        assert np.allclose(tuple(info.origin), o, atol=1e-12)
        dynamic.add_block_from_parent(ms, o, h, d)
    compare(dom, ms, "shadow scales started")
    for _ in range(2):
        dom.step(1)
        ms.step()
    compare(dom, ms, "shadow scales stepped")
    dom.close()


def test_shadow_scales_point_light_cone(lib):
    """A cube lit by one inflow node on the upstream face: with 2 scales and d = 0 the refined
    block is the bounding box of the cube and its shadow cone (the nodes that see c = 0 of
    M = 1 samples), as the oracle counts it; without obstacles nothing is added."""
    from paper_1807_02284_gb300 import lbm
    dims = (40, 24, 24)
    shape = dims[::-1]
    flags = np.zeros(shape, np.uint8)
    flags[9:15, 9:15, 10:16] = 1                     # cube x 10..15, y 9..14, z 9..14
    flags[12, 12, 0] = 2                             # one inflow node
    plan = dynamic.shadow_scales(flags, 2, 0.5, 0.0, 20.0, flow_axis=0, n_light=4)
    assert len(plan) == 1
    (o, h, d), = plan
    assert d[0] > (15 - 10) / h + 1                 # the cone reaches past the cube
    for fl, n_want in ((flags, 1), (flags & 2, 0)):
        dom = lbm.Domain(dims, 0.01)
        dom.set_flags(fl)
        dom.init_macro(np.zeros(shape + (3,), np.float32), rho=np.ones(shape, np.float32),
                       c=np.zeros(shape, np.float32))
        assert dom.build_static_scales_shadow(2, 0.5, 0.0, 20.0, 0, 4) == n_want
        if n_want:
            info = dom.info(1)
            assert tuple(info.dims) == d and abs(info.h - h) < 1e-12
            assert np.allclose(tuple(info.origin), o, atol=1e-12)
        dom.close()
