"""GPU parity of the single-block collide-stream path (pull, bounce-back, faces, inflow,
adaptive CMR collision, scalar) against the FP64 oracle, through the C-ABI.

Tolerances (FP32 path): velocity max-abs error <= 1e-5 * max|u| (the stated target);
populations max-abs error <= 2e-7 (FP32 unit roundoff 6e-8 on stored shifted populations of
magnitude <= 0.05, accumulated over the short horizons used here); scalar <= 1e-6.
"""
import math

import numpy as np
import pytest

import synth
from oracle import grid
from tests.helpers import (f32, gpu_domain, gpu_state, max_err, oracle_params, oracle_state,
                           state_from_arrays)

pytestmark = pytest.mark.gpu

U_REL = 1e-5
F_ABS = 2e-7
C_ABS = 1e-6


def _compare(dom, st, b, label=""):
    f, u, c = gpu_state(dom, b.shape_zyx)
    umax = float(np.abs(st.u.numpy()).max())
    eu = max_err(u, st.u.numpy())
    ef = max_err(f, st.f.numpy())
    ec = max_err(c, st.c.numpy())
    print(f"{label}: |du|={eu:.2e} (max|u| {umax:.3f}) |df|={ef:.2e} |dc|={ec:.2e}")
    assert eu <= U_REL * umax, f"{label} velocity error {eu:.3e}"
    assert ef <= F_ABS, f"{label} population error {ef:.3e}"
    assert ec <= C_ABS, f"{label} scalar error {ec:.3e}"


SCENES = {
    "periodic_ragged": dict(dims=(40, 37, 19), seed=1, periodic=(True, True, True)),
    "open_sphere_inflow": dict(dims=(45, 33, 21), seed=2, periodic=(False, False, False),
                               spheres=[(20.0, 16.0, 10.0, 5.5)], inflow=(16, 10, 5.0, 0.1)),
    "mixed_faces_two_spheres": dict(dims=(34, 29, 26), seed=3, periodic=(False, True, False),
                                    spheres=[(10.0, 8.0, 8.0, 3.0), (25.0, 20.0, 17.0, 4.0)],
                                    inflow=(14, 12, 4.0, 0.06)),
    "fixed_relaxation": dict(dims=(33, 17, 12), seed=4, periodic=(True, False, True),
                             adaptive=False),
}


@pytest.mark.parametrize("name", list(SCENES))
def test_parity_random_scenes(lib, name):
    sc = synth.random_scene(**SCENES[name])
    b = sc.blocks[0]
    dom = gpu_domain(sc)
    st = oracle_state(sc)
    p = oracle_params(sc)
    for n in range(8):
        dom.step(1)
        st = grid.step(st, p)
    dom.sync()
    _compare(dom, st, b, name)
    dom.close()


@pytest.mark.parametrize("name", ["open_sphere_inflow", "periodic_ragged"])
def test_parity_local_strain_relaxation(lib, name):
    """Adaptive relaxation driven by the node's own non-equilibrium strain rate."""
    sc = synth.random_scene(**SCENES[name])
    b = sc.blocks[0]
    dom = gpu_domain(sc, grad_mode="local")
    st = oracle_state(sc)
    p = oracle_params(sc, grad_mode="local")
    for n in range(8):
        dom.step(1)
        st = grid.step(st, p)
    dom.sync()
    _compare(dom, st, b, f"local strain {name}")
    dom.close()


def test_parity_far_from_equilibrium_populations(lib):
    """Arbitrary positive populations (all 27 moments away from equilibrium), random lagged
    velocity and scalar: one step."""
    from paper_1807_02284_gb300 import lbm
    sc = synth.random_scene(dims=(36, 20, 11), seed=5, periodic=(True, False, True),
                            spheres=[(18.0, 10.0, 5.0, 3.0)])
    b = sc.blocks[0]
    dom = gpu_domain(sc)
    f0 = synth.random_populations(b.shape_zyx, seed=6, eps=0.3)
    solid = (b.flags & synth.SOLID) != 0
    rng = np.random.default_rng(7)
    u_lag = f32(0.08 * (2 * rng.random((3,) + b.shape_zyx) - 1)).astype(np.float64)
    c0 = f32(rng.random(b.shape_zyx)).astype(np.float64)
    f0 = f32(f0).astype(np.float64)
    dom.write_field(lbm.LBM_FIELD_F, f0)
    dom.write_field(lbm.LBM_FIELD_U, u_lag)
    dom.write_field(lbm.LBM_FIELD_SCALAR, c0)
    dom.step(1)
    dom.sync()
    st = state_from_arrays(f0, u_lag, c0, b.flags)
    st = grid.step(st, oracle_params(sc))
    f, u, c = gpu_state(dom, b.shape_zyx)
    fluid = ~solid
    eu = max_err(u[:, fluid], st.u.numpy()[:, fluid])
    umax = float(np.abs(st.u.numpy()).max())
    print(f"far-from-eq: |du|={eu:.2e} |df|={max_err(f, st.f.numpy()):.2e}")
    assert eu <= U_REL * umax
    assert max_err(f, st.f.numpy()) <= 5e-7
    assert max_err(c, st.c.numpy()) <= C_ABS
    dom.close()


def test_taylor_green_32_parity_and_decay(lib):
    """Config 1: 32^3 periodic Taylor-Green vortex, Re = 100, adaptive relaxation, 200 steps.
    GPU vs oracle (the oracle runs the z-invariant flow on 32x32x2, identical by symmetry)
    and the GPU's mode decay rate against the closed form exp(-2 nu k^2 t)."""
    n = 32
    sc = synth.taylor_green(n)
    sc2 = synth.taylor_green(n, nz=2)
    dom = gpu_domain(sc)
    st = oracle_state(sc2)
    p = oracle_params(sc2)
    k = 2 * math.pi / n
    x = np.arange(n)
    basis = np.sin(k * x)[None, None, :] * np.cos(k * x)[None, :, None]
    amps = {}
    from paper_1807_02284_gb300 import lbm
    for t in range(1, 201):
        dom.step(1)
        st = grid.step(st, p)
        if t in (60, 200):
            u = dom.read_field(lbm.LBM_FIELD_U, lbm.LBM_F64).reshape(3, n, n, n)
            amps[t] = float((u[0] * basis).sum() / (basis * basis).sum() / n)
    f, u, c = gpu_state(dom, (n, n, n))
    eu = max_err(u[:, :2], st.u.numpy())
    umax = float(np.abs(st.u.numpy()).max())
    print(f"TGV: |du|={eu:.2e} max|u|={umax:.4f}")
    assert eu <= U_REL * umax
    assert np.abs(u[:, 0] - u[:, 17]).max() < 1e-12 + 1e-6 * umax   # z-invariance kept
    rate = -math.log(amps[200] / amps[60]) / 140.0
    assert rate == pytest.approx(2 * sc.nu * k * k, rel=5e-3)
    dom.close()


def test_reductions_match_oracle(lib):
    sc = synth.random_scene(dims=(30, 26, 22), seed=8, periodic=(False, True, True),
                            spheres=[(15.0, 13.0, 11.0, 4.0)], inflow=(13, 11, 4.0, 0.1))
    dom = gpu_domain(sc)
    st = oracle_state(sc)
    p = oracle_params(sc)
    for _ in range(4):
        dom.step(1)
        st = grid.step(st, p)
    r_gpu = dom.reduce()
    r_or = grid.reductions(st).numpy()
    print("reduce gpu", r_gpu, "oracle", r_or)
    assert abs(r_gpu[0] - r_or[0]) / r_or[0] < 1e-7
    assert np.abs(r_gpu[1:4] - r_or[1:4]).max() < 1e-5 * max(1.0, np.abs(r_or[1:4]).max())
    assert abs(r_gpu[4] - r_or[4]) / r_or[4] < 1e-5
    dom.close()


def test_mass_drift_periodic_run(lib):
    sc = synth.random_scene(dims=(64, 64, 64), seed=9, periodic=(True, True, True), nu=1e-3)
    dom = gpu_domain(sc)
    m0 = dom.reduce()[0]
    dom.step(300)
    m1 = dom.reduce()[0]
    print("mass drift", (m1 - m0) / m0)
    assert abs(m1 - m0) / m0 <= 1e-6
    dom.close()


def test_graph_replay_is_bit_identical_to_direct_launches(lib):
    from paper_1807_02284_gb300 import lbm
    sc = synth.random_scene(dims=(48, 40, 20), seed=10, periodic=(False, False, False),
                            spheres=[(24.0, 20.0, 10.0, 5.0)], inflow=(20, 10, 5.0, 0.1))
    a = gpu_domain(sc)
    b = gpu_domain(sc)
    a.step(40)                      # captured graph of 16-step chunks + direct tail
    for _ in range(40):
        b.step(1)                   # one launch per call
    fa = a.read_field(lbm.LBM_FIELD_F, lbm.LBM_F32)
    fb = b.read_field(lbm.LBM_FIELD_F, lbm.LBM_F32)
    assert np.array_equal(fa, fb)
    a.close(); b.close()


@pytest.mark.parametrize("dims,periodic", [((1, 1, 1), (True, True, True)),
                                           ((3, 1, 2), (True, False, True)),
                                           ((2, 5, 3), (False, False, False))])
def test_degenerate_small_blocks(lib, dims, periodic):
    sc = synth.random_scene(dims=dims, seed=11, periodic=periodic)
    dom = gpu_domain(sc)
    st = oracle_state(sc)
    p = oracle_params(sc)
    for _ in range(3):
        dom.step(1)
        st = grid.step(st, p)
    _compare(dom, st, sc.blocks[0], f"degenerate {dims}")
    dom.close()


def test_divergence_is_reported(lib):
    from paper_1807_02284_gb300 import lbm
    sc = synth.random_scene(dims=(16, 16, 16), seed=12)
    dom = gpu_domain(sc)
    f = dom.read_field(lbm.LBM_FIELD_F, lbm.LBM_F64).reshape(27, -1)
    f[:, 100] = np.nan
    dom.write_field(lbm.LBM_FIELD_F, f.reshape(-1))
    dom.step(1)
    with pytest.raises(lbm.LBMError) as ei:
        dom.sync()
    assert ei.value.status == lbm.LBM_ERR_DIVERGED
    # the context stays usable: re-initialise and step again
    b = sc.blocks[0]
    dom.init_macro(f32(b.u0), rho=f32(b.rho0), c=f32(b.c0))
    dom.step(2)
    dom.sync()
    dom.close()


def test_host_side_argument_errors(lib):
    from paper_1807_02284_gb300 import lbm
    sc = synth.random_scene(dims=(8, 8, 8), seed=13)
    dom = gpu_domain(sc)
    with pytest.raises(lbm.LBMError) as ei:
        dom.read_field(lbm.LBM_FIELD_U, lbm.LBM_F32, block=3)
    assert ei.value.status == lbm.LBM_ERR_INVALID_ARG
    with pytest.raises(lbm.LBMError):
        dom.set_flags(np.zeros(10, np.uint8))          # too short
    with pytest.raises(lbm.LBMError) as ei:
        dom.step(-1)
    assert ei.value.status == lbm.LBM_ERR_INVALID_ARG
    # an inflow record outside the block is skipped and reported
    rec = np.zeros(1, dtype=lbm.INFLOW_RECORD)
    rec["x"] = 99
    dom.set_inflow(rec)
    with pytest.raises(lbm.LBMError) as ei:
        dom.sync()
    assert ei.value.status == lbm.LBM_ERR_DIVERGED
    dom.close()
