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


def _reference(f, flags, N):
    """Mass, momentum and kinetic energy of non-obstacle, non-ghost nodes, in FP64 from the
    definitions (rho = sum f, j = sum c f over the paper's velocity list)."""
    from oracle import cmr
    f = f.view(27, N).double()
    keep = (flags & 9) == 0
    rho = f.sum(0)
    j = cmr.C.to(f.device).T @ f
    return np.array([float(rho[keep].sum()), *(float(j[a][keep].sum()) for a in range(3)),
                     float((0.5 * (j * j).sum(0) / rho)[keep].sum())])


def test_noalloc_reduce_many_partials_between_small_calls(lib):
    """A 128^3 field (128 per-CTA partials) between two small calls (3 partials): no call
    depends on what an earlier call of another size left in the shared scratch."""
    from oracle import cmr
    from paper_1807_02284_gb300 import lbm
    stream = torch.cuda.current_stream()
    w = cmr.equilibrium(torch.ones(1, dtype=torch.float64),
                        torch.zeros(1, 3, dtype=torch.float64))[0].cuda()
    out = torch.empty(5, dtype=torch.float64, device="cuda")
    g = torch.Generator(device="cuda").manual_seed(7)
    for n in (40 * 36 * 30, 128 ** 3, 40 * 36 * 30):
        f = (w[:, None] * (1.0 + 0.02 * (2 * torch.rand(27, n, generator=g, device="cuda",
                                                       dtype=torch.float64) - 1))).contiguous()
        flags = (torch.rand(n, generator=g, device="cuda") < 0.05).to(torch.uint8)
        flags[::97] |= 8
        ref = _reference(f, flags, n)
        for dt, arr in ((lbm.LBM_F64, f), (lbm.LBM_F32, f.float())):
            out.fill_(float("nan"))
            st = lib.lbm_reduce_noalloc(C.c_void_p(arr.data_ptr()), dt,
                                        C.c_void_p(flags.data_ptr()), n,
                                        C.c_void_p(out.data_ptr()), C.c_void_p(stream.cuda_stream))
            assert st == lbm.LBM_OK
            torch.cuda.synchronize()
            _check(out.cpu().numpy(), ref)
