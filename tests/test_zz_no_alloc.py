"""lbm_reduce_noalloc: the diagnostics reduction for callers that cannot allocate device
memory (for example a process whose device memory belongs to another framework's pool).

It keeps its partial sums in a fixed array inside the library instead of allocating, so it
must give the same mass, momentum and kinetic energy as lbm_reduce on the same state, call
after call.  This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest
import torch

import synth
from tests.helpers import gpu_domain

pytestmark = pytest.mark.gpu


def _check(got, ref):
    # the tolerances of the oracle reduction test
    assert abs(got[0] - ref[0]) / ref[0] < 1e-7
    assert np.abs(got[1:4] - ref[1:4]).max() < 1e-5 * max(1.0, np.abs(ref[1:4]).max())
    assert abs(got[4] - ref[4]) / ref[4] < 1e-5


def test_noalloc_reduce_matches_lbm_reduce_on_consecutive_calls(lib):
    from paper_1807_02284_gb300 import lbm
    sc = synth.random_scene(dims=(40, 36, 30), seed=31, periodic=(False, True, True),
                            spheres=[(20.0, 18.0, 15.0, 5.0)], inflow=(18, 15, 4.0, 0.1))
    dom = gpu_domain(sc)
    N = sc.blocks[0].flags.size
    stream = torch.cuda.current_stream()
    out = torch.empty(5, dtype=torch.float64, device="cuda")
    for call in range(2):
        dom.step(3)
        ref = dom.reduce()
        f = torch.empty(27 * N, dtype=torch.float64, device="cuda")
        flags = torch.empty(N, dtype=torch.uint8, device="cuda")
        dom.read_field(lbm.LBM_FIELD_F, lbm.LBM_F64, out=f)
        dom.read_field(lbm.LBM_FIELD_FLAGS, lbm.LBM_U8, out=flags)
        out.fill_(float("nan"))
        st = lib.lbm_reduce_noalloc(C.c_void_p(f.data_ptr()), lbm.LBM_F64,
                                    C.c_void_p(flags.data_ptr()), N,
                                    C.c_void_p(out.data_ptr()), C.c_void_p(stream.cuda_stream))
        assert st == lbm.LBM_OK, lib.lbm_last_error(None)
        torch.cuda.synchronize()
        _check(out.cpu().numpy(), ref)
        # float32 input gives the same result within the same tolerance
        f32 = f.float()
        st = lib.lbm_reduce_noalloc(C.c_void_p(f32.data_ptr()), lbm.LBM_F32,
                                    C.c_void_p(flags.data_ptr()), N,
                                    C.c_void_p(out.data_ptr()), C.c_void_p(stream.cuda_stream))
        assert st == lbm.LBM_OK
        torch.cuda.synchronize()
        _check(out.cpu().numpy(), ref)
    dom.close()


def test_noalloc_reduce_rejects_sizes_beyond_its_scratch(lib):
    from paper_1807_02284_gb300 import lbm
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    st = lib.lbm_reduce_noalloc(C.c_void_p(dummy.data_ptr()), lbm.LBM_F64, None,
                                lbm.LBM_REDUCE_NOALLOC_MAX_NODES + 1,
                                C.c_void_p(dummy.data_ptr()), None)
    assert st == lbm.LBM_ERR_INVALID_ARG
    assert b"n_nodes" in lib.lbm_last_error(None)
