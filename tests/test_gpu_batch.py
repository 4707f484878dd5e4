"""Batched persistent stepping (one cooperative launch per call over the joint work list of
many domains of uneven sizes): bit-identical to stepping each domain alone, parity with the
oracle, and the bounded device barrier reporting a timeout instead of hanging."""
import numpy as np
import pytest

import synth
from oracle import grid
from tests.helpers import gpu_domain, gpu_state, max_err, oracle_params, oracle_state

pytestmark = pytest.mark.gpu


def _scenes(count, seed, lo=12, hi=40):
    return synth.batch(count=count, seed=seed, lo=lo, hi=hi, nu=2e-3)


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_batch_is_bit_identical_to_single_domain_steps(lib, storage):
    from paper_1807_02284_gb300 import lbm
    scenes = _scenes(9, seed=40)
    batched = [gpu_domain(s, storage) for s in scenes]
    single = [gpu_domain(s, storage) for s in scenes]
    for steps in (6, 5):                      # even and odd step counts (level parity)
        lbm.step_batch(batched, steps)
        for d in single:
            d.step(steps)
    for a, b in zip(batched, single):
        fa = a.read_field(lbm.LBM_FIELD_F, lbm.LBM_F32)
        fb = b.read_field(lbm.LBM_FIELD_F, lbm.LBM_F32)
        assert np.array_equal(fa, fb)
        assert np.array_equal(a.read_field(lbm.LBM_FIELD_SCALAR, lbm.LBM_F32),
                              b.read_field(lbm.LBM_FIELD_SCALAR, lbm.LBM_F32))
        assert a.info().steps == 11
    for d in batched + single:
        d.close()


def test_batch_single_steps_reuse_plans_and_stay_identical(lib):
    """Repeated one-step calls flip every member's level each time (two cached plans in
    turn); a member destroyed and replaced between calls must not be stepped through a stale
    plan.  Results stay bit-identical to single-domain stepping."""
    from paper_1807_02284_gb300 import lbm
    scenes = _scenes(5, seed=42)
    batched = [gpu_domain(s) for s in scenes]
    single = [gpu_domain(s) for s in scenes]
    for _ in range(5):
        lbm.step_batch(batched, 1)
        for d in single:
            d.step(1)
    batched[2].close()
    single[2].close()
    batched[2] = gpu_domain(scenes[2])
    single[2] = gpu_domain(scenes[2])
    for _ in range(3):
        lbm.step_batch(batched, 1)
        for d in single:
            d.step(1)
    for a, b in zip(batched, single):
        assert np.array_equal(a.read_field(lbm.LBM_FIELD_F, lbm.LBM_F32),
                              b.read_field(lbm.LBM_FIELD_F, lbm.LBM_F32))
    for d in batched + single:
        d.close()


def test_reduce_batch_equals_per_domain_reduce(lib):
    from paper_1807_02284_gb300 import lbm
    scenes = _scenes(6, seed=43)
    doms = [gpu_domain(s) for s in scenes]
    lbm.step_batch(doms, 7)
    r = lbm.reduce_batch(doms)
    assert r.shape == (6, 5)
    # members on streams of their own: one reduction each, the very values of lbm_reduce
    for i, d in enumerate(doms):
        assert np.array_equal(r[i], d.reduce())
    # members sharing a stream: one launch over all of them, the same sums in another order
    # (per-thread compensated FP32 partials over other nodes, FP64 combination)
    import torch
    from tests.helpers import f32
    st = torch.cuda.Stream()
    shared = []
    for s in scenes:
        b = s.blocks[0]
        d = lbm.Domain(b.dims, s.nu, periodic=s.periodic, adaptive=s.adaptive, c_src=s.c_src,
                       stream=st)
        d.set_flags(b.flags)
        d.init_macro(f32(b.u0), rho=f32(b.rho0), c=f32(b.c0))
        shared.append(d)
    lbm.step_batch(shared, 7)
    r2 = lbm.reduce_batch(shared)
    for i, d in enumerate(shared):
        ri = d.reduce()
        assert abs(r2[i][0] - ri[0]) <= 1e-9 * ri[0]
        assert np.abs(r2[i][1:] - ri[1:]).max() <= 1e-6 * max(1.0, np.abs(ri[1:]).max())
        assert np.array_equal(ri, r[i])             # same states as the separate-stream run
    for d in shared:
        d.close()
    with pytest.raises(lbm.LBMError) as ei:
        lbm.reduce_batch(doms, block=1)
    assert ei.value.status == lbm.LBM_ERR_INVALID_ARG
    for d in doms:
        d.close()


def test_batch_matches_oracle(lib):
    from paper_1807_02284_gb300 import lbm
    scenes = _scenes(4, seed=41, lo=10, hi=22)
    doms = [gpu_domain(s) for s in scenes]
    lbm.step_batch(doms, 4)
    for d, s in zip(doms, scenes):
        st = oracle_state(s)
        p = oracle_params(s)
        for _ in range(4):
            st = grid.step(st, p)
        f, u, c = gpu_state(d, s.blocks[0].shape_zyx)
        umax = float(np.abs(st.u.numpy()).max())
        eu = max_err(u, st.u.numpy())
        print(f"batch {s.name}: |du|={eu:.2e} max|u|={umax:.3f}")
        assert eu <= 1e-5 * umax
        assert max_err(f, st.f.numpy()) <= 2e-7
        d.close()


def test_batch_full_size_sixty_four_simulations(lib):
    """The 64-simulation workload (edges 24..96): one call of 30 steps equals 30 single
    steps of a few sampled members, and stays finite everywhere."""
    from paper_1807_02284_gb300 import lbm
    scenes = synth.batch(64, seed=4)
    doms = [gpu_domain(s) for s in scenes]
    lbm.step_batch(doms, 30)
    for i in (0, 17, 63):
        ref = gpu_domain(scenes[i])
        ref.step(30)
        assert np.array_equal(doms[i].read_field(lbm.LBM_FIELD_U, lbm.LBM_F32),
                              ref.read_field(lbm.LBM_FIELD_U, lbm.LBM_F32))
        ref.close()
    for d in doms:
        d.sync()
        d.close()


def test_batch_argument_checks(lib):
    from paper_1807_02284_gb300 import lbm
    a = lbm.Domain((8, 8, 8), 1e-3)
    b = lbm.Domain((8, 8, 8), 1e-3, storage="fp16")
    with pytest.raises(lbm.LBMError) as ei:
        lbm.step_batch([a, b], 2)
    assert ei.value.status == lbm.LBM_ERR_INVALID_ARG
    with pytest.raises(lbm.LBMError):
        lbm.step_batch([a, a], 2)
    c = lbm.Domain((16, 16, 16), 1e-3)
    c.add_scale_block((2, 2, 2), 0.5, (8, 8, 8))
    with pytest.raises(lbm.LBMError) as ei:
        lbm.step_batch([a, c], 2)
    assert ei.value.status == lbm.LBM_ERR_UNSUPPORTED
    for d in (a, b, c):
        d.close()


def test_bounded_barrier_reports_timeout_and_context_survives(lib):
    from paper_1807_02284_gb300 import lbm
    assert lib.lbm_barrier_selftest(0, 100.0, None) == lbm.LBM_OK
    assert lib.lbm_barrier_selftest(1, 20.0, None) == lbm.LBM_ERR_TIMEOUT
    # the context is still usable afterwards
    s = synth.random_scene(dims=(12, 12, 12), seed=5)
    d = gpu_domain(s)
    d.step(2)
    d.sync()
    d.close()


def test_set_inflow_batch_equals_per_member_calls(lib):
    """One staged upload and launch for the inflow records of members sharing a stream: the
    same flags, velocity levels and populations as for members on their own streams (which
    take the per-member lbm_set_boundary calls), and a bad record is reported by its own
    member only."""
    import torch
    from paper_1807_02284_gb300 import lbm
    from tests.helpers import f32
    scenes = _scenes(5, seed=44)
    st = torch.cuda.Stream()
    joint, single = [], []
    for s in scenes:
        b = s.blocks[0]
        d = lbm.Domain(b.dims, s.nu, periodic=s.periodic, adaptive=s.adaptive, c_src=s.c_src,
                       stream=st)
        d.set_flags(b.flags)
        d.init_macro(f32(b.u0), rho=f32(b.rho0), c=f32(b.c0))
        joint.append(d)
        single.append(gpu_domain(s))
    rng = np.random.default_rng(7)
    recs = []
    for s in scenes:
        r = synth.inflow_records(s.blocks[0])
        r["ux"] *= (1.0 + 0.05 * rng.random(r.size)).astype(np.float32)
        recs.append(r)
    recs[2] = recs[2][:0]                           # a member without records
    lbm.set_inflow_batch(joint, recs)                # one staged upload and launch
    lbm.set_inflow_batch(single, recs)               # own streams: the per-member calls
    lbm.step_batch(joint, 3)
    lbm.step_batch(single, 3)
    for a, b in zip(joint, single):
        for field, dt in ((lbm.LBM_FIELD_U, lbm.LBM_F32), (lbm.LBM_FIELD_FLAGS, lbm.LBM_U8),
                          (lbm.LBM_FIELD_F, lbm.LBM_F32)):
            assert np.array_equal(a.read_field(field, dt), b.read_field(field, dt))
    bad = synth.inflow_records(scenes[1].blocks[0])[:1].copy()
    bad["x"] = 10_000                               # outside member 1's block
    lbm.set_inflow_batch(joint, [recs[0][:0], bad, recs[2], recs[3][:0], recs[4][:0]])
    with pytest.raises(lbm.LBMError) as ei:
        joint[1].sync()
    assert ei.value.status == lbm.LBM_ERR_DIVERGED
    joint[0].sync()
    for d in joint + single:
        d.close()


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_step_batch_reduce_state_and_values(lib, storage):
    """lbm_step_batch_reduce: the states of lbm_step_batch, and every member's diagnostics
    within FP32 rounding of lbm_reduce's (FP16: of the FP32 state before its rounding)."""
    from paper_1807_02284_gb300 import lbm
    scenes = _scenes(6, seed=45)
    a = [gpu_domain(s, storage) for s in scenes]
    b = [gpu_domain(s, storage) for s in scenes]
    r = lbm.step_batch_reduce(a, 5)
    lbm.step_batch(b, 5)
    tol_m, tol_j = (1e-7, 1e-5) if storage == "fp32" else (1e-5, 1e-3)
    for i, (x, y) in enumerate(zip(a, b)):
        assert np.array_equal(x.read_field(lbm.LBM_FIELD_F, lbm.LBM_F32),
                              y.read_field(lbm.LBM_FIELD_F, lbm.LBM_F32))
        ri = y.reduce()
        assert abs(r[i][0] - ri[0]) <= tol_m * ri[0]
        assert np.abs(r[i][1:] - ri[1:]).max() <= tol_j * max(1.0, np.abs(ri[1:]).max())
    for k in range(3):                                   # single steps, both level parities
        r = lbm.step_batch_reduce(a, 1)
        lbm.step_batch(b, 1)
        for i, y in enumerate(b):
            ri = y.reduce()
            assert abs(r[i][0] - ri[0]) <= tol_m * ri[0]
    with pytest.raises(lbm.LBMError) as ei:
        lbm.step_batch_reduce(a, 0)
    assert ei.value.status == lbm.LBM_ERR_INVALID_ARG
    for d in a + b:
        d.close()


def test_step_batch_reduce_async_equals_sync(lib):
    """lbm_step_batch_reduce_async pipelined (the next batched step queued before the previous
    diagnostics are waited for) gives the states of the same sequence of lbm_step_batch_reduce
    calls bit for bit and their diagnostics to FP32 rounding (the two domain sets tune their
    work-item sizes separately, so their per-item partial sums may be cut differently); its
    tickets come from the first domain's sequence."""
    import torch
    from paper_1807_02284_gb300 import lbm
    scenes = _scenes(6, seed=47)
    a = [gpu_domain(s) for s in scenes]
    b = [gpu_domain(s) for s in scenes]
    out = torch.zeros((5, len(b), 5), dtype=torch.float64, pin_memory=True)
    ref, got, tickets = [], [], []
    for k in range(5):
        ref.append(lbm.step_batch_reduce(a, 1 + k % 2))
        tickets.append(lbm.step_batch_reduce_async(b, 1 + k % 2, out[k]))
        if k:
            b[0].wait_results(tickets[k - 1])
            got.append(out[k - 1].numpy().copy())
    b[0].wait_results(tickets[-1])
    got.append(out[4].numpy().copy())
    assert tickets == list(range(1, 6))
    for x, y in zip(ref, got):
        assert np.abs(x[:, 0] - y[:, 0]).max() <= 1e-7 * np.abs(x[:, 0]).max()
        assert np.abs(x[:, 1:] - y[:, 1:]).max() <= 1e-5 * max(1.0, np.abs(x[:, 1:]).max())
    for x, y in zip(a, b):
        assert np.array_equal(x.read_field(lbm.LBM_FIELD_F, lbm.LBM_F32),
                              y.read_field(lbm.LBM_FIELD_F, lbm.LBM_F32))
    with pytest.raises(lbm.LBMError) as ei:
        lbm.step_batch_reduce_async(b, 0, out[0])
    assert ei.value.status == lbm.LBM_ERR_INVALID_ARG
    for d in a + b:
        d.close()
