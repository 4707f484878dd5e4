"""The two-node collide-stream kernel (k_step2: nodes x, x + 1 of a row per thread, paired
FP32 arithmetic) against the one-node kernel and the FP64 oracle, through the C-ABI.

The launch shape is forced with LBM_TILE ("bx,by,code": code 3 or 4 = one-node kernel,
20, 21 or 22 = two-node kernel with 4, 5 or 6 CTAs per SM), read when a block is created.
Every launch shape computes the same values, so the two kernels must agree bit for bit on
populations, velocity and scalar, for every kind of node the pair path hands back to the
one-node update (obstacle voxels and their neighbours, inflow, faces, walls, scalar
sources) and for both storage types and gradient modes."""
import numpy as np
import pytest

import synth
from oracle import grid
from tests.helpers import gpu_domain, gpu_state, max_err, oracle_params, oracle_state

pytestmark = pytest.mark.gpu

ONE_NODE, PAIR4, PAIR5, PAIR6 = "64,4,3", "64,4,20", "128,2,21", "256,1,22"

SCENES = {
    "open_sphere_inflow": dict(dims=(46, 33, 21), seed=2, periodic=(False, False, False),
                               spheres=[(20.0, 16.0, 10.0, 5.5)], inflow=(16, 10, 5.0, 0.1)),
    "periodic": dict(dims=(40, 37, 19), seed=1, periodic=(True, True, True)),
    "mixed_faces": dict(dims=(34, 29, 26), seed=3, periodic=(True, False, False),
                        spheres=[(10.0, 8.0, 8.0, 3.0), (25.0, 20.0, 17.0, 4.0)],
                        inflow=(14, 12, 4.0, 0.06)),
    "fixed_relaxation": dict(dims=(66, 17, 12), seed=4, periodic=(False, False, True),
                             adaptive=False),
}


def _run(monkeypatch, tile, sc, steps, storage="fp32", grad_mode="lagged", walls=None,
         obstacle_walls=False):
    from paper_1807_02284_gb300 import lbm
    monkeypatch.setenv("LBM_TILE", tile)
    dom = gpu_domain(sc, storage=storage, grad_mode=grad_mode)
    if walls is not None:
        dom.set_walls(walls, obstacles=obstacle_walls)
    info = dom.info(0)
    dom.step(steps)
    dom.sync()
    shape = sc.blocks[0].shape_zyx
    f, u, c = gpu_state(dom, shape, dtype=lbm.LBM_F32)
    dom.close()
    return info, f, u, c


def _assert_identical(a, b, label):
    for name, x, y in zip("fuc", a[1:], b[1:]):
        assert np.array_equal(x, y), f"{label}: {name} differs (max {max_err(x, y):.3e})"


def _with_scalar_sources(sc, seed):
    """Marks a seeded tenth of the fluid nodes as scalar sources."""
    b = sc.blocks[0]
    rng = np.random.default_rng(seed)
    fluid = (b.flags & (synth.SOLID | synth.INFLOW)) == 0
    pick = fluid & (rng.random(b.shape_zyx) < 0.1)
    b.flags[pick] |= synth.SCALAR_SRC
    return sc


@pytest.mark.parametrize("name", list(SCENES))
@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_pair_kernel_is_bit_identical(lib, monkeypatch, name, storage):
    sc = _with_scalar_sources(synth.random_scene(**SCENES[name]), 7)
    ref = _run(monkeypatch, ONE_NODE, sc, 6, storage)
    assert ref[0].nodes_per_thread == 1 and ref[0].ctas_per_sm == 3
    for tile, bound in ((PAIR4, 4), (PAIR5, 5), (PAIR6, 6)):
        got = _run(monkeypatch, tile, sc, 6, storage)
        assert got[0].nodes_per_thread == 2 and got[0].ctas_per_sm == bound
        _assert_identical(ref, got, f"{name} {storage} {tile}")


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_pair_kernel_local_strain_is_bit_identical(lib, monkeypatch, storage):
    sc = synth.random_scene(**SCENES["open_sphere_inflow"])
    ref = _run(monkeypatch, ONE_NODE, sc, 6, storage, grad_mode="local")
    got = _run(monkeypatch, PAIR4, sc, 6, storage, grad_mode="local")
    _assert_identical(ref, got, f"local strain {storage}")


@pytest.mark.parametrize("obstacles", [False, True])
def test_pair_kernel_with_walls_is_bit_identical(lib, monkeypatch, obstacles):
    sc = synth.random_scene(dims=(26, 22, 18), seed=51, periodic=(False, False, False),
                            spheres=[(13.0, 11.0, 9.0, 3.0)], inflow=(11, 9, 3.0, 0.07), nu=0.01)
    walls = (False, True, True, True, True, True)
    ref = _run(monkeypatch, ONE_NODE, sc, 6, walls=walls, obstacle_walls=obstacles)
    got = _run(monkeypatch, PAIR4, sc, 6, walls=walls, obstacle_walls=obstacles)
    _assert_identical(ref, got, f"walls, obstacle walls {obstacles}")


def test_odd_x_extent_falls_back_to_one_node(lib, monkeypatch):
    """An odd nx has no aligned pairs: the two-node code runs the one-node kernel."""
    sc = synth.random_scene(dims=(45, 20, 14), seed=9, periodic=(False, True, False),
                            spheres=[(20.0, 10.0, 7.0, 3.5)])
    ref = _run(monkeypatch, ONE_NODE, sc, 4)
    got = _run(monkeypatch, PAIR4, sc, 4)
    assert got[0].nodes_per_thread == 1
    _assert_identical(ref, got, "odd nx")


def test_pair_kernel_matches_oracle(lib, monkeypatch):
    """Direct parity of the two-node kernel with the FP64 oracle (same bounds as the
    one-node parity tests: velocity 1e-5 max|u|, populations 2e-7, scalar 1e-6)."""
    sc = _with_scalar_sources(synth.random_scene(**SCENES["open_sphere_inflow"]), 11)
    b = sc.blocks[0]
    monkeypatch.setenv("LBM_TILE", PAIR4)
    dom = gpu_domain(sc)
    st, p = oracle_state(sc), oracle_params(sc)
    for _ in range(8):
        dom.step(1)
        st = grid.step(st, p)
    f, u, c = gpu_state(dom, b.shape_zyx)
    dom.close()
    umax = float(np.abs(st.u.numpy()).max())
    eu, ef, ec = max_err(u, st.u.numpy()), max_err(f, st.f.numpy()), max_err(c, st.c.numpy())
    print(f"pair kernel: |du|={eu:.2e} (max|u| {umax:.3f}) |df|={ef:.2e} |dc|={ec:.2e}")
    assert eu <= 1e-5 * umax and ef <= 2e-7 and ec <= 1e-6


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
@pytest.mark.parametrize("walls", [False, True])
def test_pair_step_reduce_is_bit_identical(lib, monkeypatch, storage, walls):
    """lbm_step_reduce with the two-node fused-diagnostics kernel: on the same node tile it
    writes the same CTA records as the one-node kernel, so the five values and the stored
    state agree bit for bit (the records, and so the last bits of the values, follow the
    tile; the state does not)."""
    from paper_1807_02284_gb300 import lbm
    sc = _with_scalar_sources(synth.random_scene(**SCENES["open_sphere_inflow"]), 5)

    def run(tile):
        monkeypatch.setenv("LBM_TILE", tile)
        dom = gpu_domain(sc, storage=storage)
        if walls:
            dom.set_walls((False, False, True, True, True, True), obstacles=True)
        vals = [dom.step_reduce(2), dom.step_reduce(1)]
        f, u, c = gpu_state(dom, sc.blocks[0].shape_zyx, dtype=lbm.LBM_F32)
        dom.close()
        return vals, (f, u, c)

    for one, pair in ((ONE_NODE, PAIR4), ("128,2,4", PAIR5)):
        ref, got = run(one), run(pair)
        for a, b in zip(ref[0], got[0]):
            assert np.array_equal(a, b), f"{pair}: {a} vs {b}"
        for name, x, y in zip("fuc", ref[1], got[1]):
            assert np.array_equal(x, y), f"{pair}: {name} differs"
