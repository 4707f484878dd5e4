"""lbm_step_reduce (the diagnostics summed by the last step's own kernel) through the C-ABI:
the stored state is the one lbm_step writes, and the five values match the FP64 oracle's
reductions of the same state and lbm_reduce (FP32 per-node terms), for FP32 and FP16-shifted
storage, wall faces and obstacle walls; multi-block domains take lbm_reduce exactly."""
import numpy as np
import pytest

import synth
from oracle import grid
from tests.helpers import gpu_domain, oracle_params, oracle_state

pytestmark = pytest.mark.gpu


def _scene(periodic=(False, True, True)):
    return synth.random_scene(dims=(30, 26, 22), seed=8, periodic=periodic,
                              spheres=[(15.0, 13.0, 11.0, 4.0)], inflow=(13, 11, 4.0, 0.1))


def _check(r, ref, mass_rtol, mom_atol, e_rtol):
    assert abs(r[0] - ref[0]) / ref[0] < mass_rtol
    assert np.abs(r[1:4] - ref[1:4]).max() < mom_atol
    assert abs(r[4] - ref[4]) / ref[4] < e_rtol


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_step_reduce_state_and_values(lib, storage):
    from paper_1807_02284_gb300 import lbm
    sc = _scene()
    b = sc.blocks[0]
    d1, d2 = gpu_domain(sc, storage), gpu_domain(sc, storage)
    d1.step(5)
    r1 = d1.reduce()
    r2 = d2.step_reduce(5)
    f1 = d1.read_field(lbm.LBM_FIELD_F, lbm.LBM_F32)
    f2 = d2.read_field(lbm.LBM_FIELD_F, lbm.LBM_F32)
    assert np.array_equal(f1, f2)                     # the step itself is unchanged
    print(storage, "reduce", r1, "step_reduce", r2)
    if storage == "fp32":
        _check(r2, r1, 1e-7, 1e-5 * max(1.0, np.abs(r1[1:4]).max()), 1e-5)
        st = oracle_state(sc)
        p = oracle_params(sc)
        for _ in range(5):
            st = grid.step(st, p)
        _check(r2, grid.reductions(st).numpy(), 1e-7, 1e-5 * max(1.0, np.abs(r1[1:4]).max()), 1e-5)
    else:   # the fused values are those of the FP32 state before its rounding for storage
        _check(r2, r1, 1e-5, 1e-3 * max(1.0, np.abs(r1[1:4]).max()), 1e-3)
    # repeated single steps keep agreeing
    for _ in range(3):
        d1.step(1)
        r1 = d1.reduce()
        r2 = d2.step_reduce(1)
        _check(r2, r1, 1e-5, 1e-3 * max(1.0, np.abs(r1[1:4]).max()), 1e-3)
    d1.close()
    d2.close()


def test_step_reduce_with_walls(lib):
    from paper_1807_02284_gb300 import lbm
    sc = _scene(periodic=(False, False, False))
    d1, d2 = gpu_domain(sc), gpu_domain(sc)
    for d in (d1, d2):
        d.set_walls((False, False, False, False, True, True), obstacles=True)
    d1.step(4)
    r1 = d1.reduce()
    r2 = d2.step_reduce(4)
    assert np.array_equal(d1.read_field(lbm.LBM_FIELD_F, lbm.LBM_F32),
                          d2.read_field(lbm.LBM_FIELD_F, lbm.LBM_F32))
    _check(r2, r1, 1e-7, 1e-5 * max(1.0, np.abs(r1[1:4]).max()), 1e-5)
    d1.close()
    d2.close()


def test_step_reduce_multiblock_is_step_then_reduce(lib):
    from tests.test_gpu_multiscale import gpu_multiscale
    sc = synth.multiscale(scale=0.25, nu=2e-3, flow_amp=0.06)
    d1, d2 = gpu_multiscale(sc), gpu_multiscale(sc)
    d1.step(2)
    r1 = d1.reduce(0)
    r2 = d2.step_reduce(2)
    assert np.array_equal(r1, r2)
    d1.close()
    d2.close()


def test_step_reduce_argument_checks(lib):
    from paper_1807_02284_gb300 import lbm
    dom = gpu_domain(_scene())
    with pytest.raises(lbm.LBMError) as ei:
        dom.step_reduce(0)
    assert ei.value.status == lbm.LBM_ERR_INVALID_ARG
    dom.step_reduce(1)
    dom.close()


@pytest.mark.parametrize("multiblock", [False, True])
def test_step_reduce_async_equals_step_reduce(lib, multiblock):
    """lbm_step_reduce_async, pipelined the way a streaming caller uses it (inflow upload
    and the next step queued before the previous diagnostics are read, pinned outputs),
    gives bit for bit the values and the state of the same sequence of lbm_step_reduce
    calls; the multi-block fallback (steps, then the separate reduction) likewise."""
    import torch
    from paper_1807_02284_gb300 import lbm
    if multiblock:
        from tests.test_gpu_multiscale import gpu_multiscale
        sc = synth.multiscale(scale=0.25, nu=2e-3, flow_amp=0.06)
        d1, d2 = gpu_multiscale(sc), gpu_multiscale(sc)
    else:
        sc = _scene(periodic=(False, False, False))
        d1, d2 = gpu_domain(sc), gpu_domain(sc)
    recs = synth.inflow_records(sc.blocks[0])
    ref, got, tickets = [], [], []
    out = torch.zeros((6, 5), dtype=torch.float64, pin_memory=True)
    for i in range(6):
        r = recs.copy()
        r["ux"] *= np.float32(1.0 + 0.01 * i)
        d1.set_inflow(r)
        ref.append(d1.step_reduce(1 + i % 2))
        d2.set_inflow(r)
        tickets.append(d2.step_reduce_async(1 + i % 2, out[i]))
        if i > 0:
            d2.wait_results(tickets[i - 1])
            got.append(out[i - 1].numpy().copy())
    d2.wait_results(tickets[-1])
    got.append(out[5].numpy().copy())
    assert tickets == list(range(1, 7))
    for a, b in zip(ref, got):
        assert np.array_equal(a, b), (a, b)
    assert np.array_equal(d1.read_field(lbm.LBM_FIELD_F, lbm.LBM_F32),
                          d2.read_field(lbm.LBM_FIELD_F, lbm.LBM_F32))
    with pytest.raises(lbm.LBMError) as ei:          # a ticket this domain has not issued
        d2.wait_results(7)
    assert ei.value.status == lbm.LBM_ERR_INVALID_ARG
    with pytest.raises(lbm.LBMError) as ei:
        d2.step_reduce_async(0, out[0])
    assert ei.value.status == lbm.LBM_ERR_INVALID_ARG
    d1.close()
    d2.close()
