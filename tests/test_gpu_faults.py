"""Failure injection on the host (no GPU fault is ever provoked): a caller allocator that
refuses the k-th device allocation, for every k a full domain life cycle makes.  Each call
must return LBM_ERR_OOM (never crash or launch on a missing buffer), the domain must stay
usable or destroyable, and every buffer the library obtained must be given back."""
import ctypes as C

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


class FailingAllocator:
    """Device memory from the torch caching allocator; allocation number `fail_at` fails."""

    def __init__(self, fail_at):
        from paper_1807_02284_gb300 import lbm
        self.fail_at = fail_at
        self.count = 0
        self.live = {}
        self.stream = torch.cuda.current_stream()

        def _alloc(nbytes, ctx):
            k = self.count
            self.count += 1
            if k == self.fail_at:
                return None
            p = torch.cuda.caching_allocator_alloc(int(nbytes), 0, self.stream)
            self.live[p] = int(nbytes)
            return p

        def _free(p, nbytes, ctx):
            assert self.live.pop(p) == int(nbytes)
            torch.cuda.caching_allocator_delete(p)

        self.fa = lbm.ALLOC_FN(_alloc)
        self.ff = lbm.FREE_FN(_free)
        self.struct = lbm.lbm_allocator(self.fa, self.ff, None)


def _life_cycle(alloc):
    """Create a 2-block domain, set flags and inflow, initialise, step (graph capture), read
    fields, reduce, then record a tape on a single-block periodic domain and run its
    adjoint.  Returns the first non-OK status (or OK) and checks that nothing leaks."""
    from paper_1807_02284_gb300 import lbm
    lib = lbm.load()
    sc = synth.multiscale(seed=2, sphere_seed=3, scale=0.125, flow_amp=0.02)
    b0 = sc.blocks[0]
    d = lbm.lbm_domain_desc()
    lib.lbm_default_desc(C.byref(d))
    d.dims[:] = list(b0.dims)
    d.nu = sc.nu
    d.cuda_stream = C.c_void_p(alloc.stream.cuda_stream)
    d.alloc = alloc.struct
    h = C.c_void_p()
    st = lib.lbm_create_domain(C.byref(d), C.byref(h))
    if st != lbm.LBM_OK:
        assert not alloc.live, "a failed creation leaked device buffers"
        return st
    first = lbm.LBM_OK

    def note(s):
        nonlocal first
        if s != lbm.LBM_OK and first == lbm.LBM_OK:
            first = s
        return s == lbm.LBM_OK

    bid = C.c_int32()
    b1 = sc.blocks[1]
    ok = note(lib.lbm_add_scale_block(h, (C.c_double * 3)(*b1.origin), b1.h,
                                      (C.c_int32 * 3)(*b1.dims), C.byref(bid)))
    nb = 2 if ok else 1
    for i in range(nb):
        blk = sc.blocks[i]
        fl = np.ascontiguousarray(blk.flags, dtype=np.uint8)
        note(lib.lbm_set_boundary(h, i, lbm.LBM_BC_FLAGS, fl.ctypes.data, fl.nbytes, 0))
        u = np.ascontiguousarray(blk.u0, dtype=np.float32)
        note(lib.lbm_init_macro(h, i, None, u.ctypes.data, None, 0))
    rec = synth.inflow_records(b0)
    note(lib.lbm_set_boundary(h, 0, lbm.LBM_BC_INFLOW, rec.ctypes.data, rec.nbytes, 0))
    note(lib.lbm_step(h, 20))
    note(lib.lbm_sync(h))
    out = np.empty(3 * b0.flags.size, np.float32)
    note(lib.lbm_read_field(h, 0, lbm.LBM_FIELD_U, lbm.LBM_F32, out.ctypes.data, out.nbytes, 0))
    red = (C.c_double * 5)()
    note(lib.lbm_reduce(h, 0, red))
    lib.lbm_destroy_domain(h)
    assert not alloc.live, f"{len(alloc.live)} device buffers leaked"
    if first != lbm.LBM_OK:
        return first
    # adjoint on a small periodic block
    sa, _ = synth.adjoint_scene(n=8, seed=5, nu=0.01, amp=0.05)
    ba = sa.blocks[0]
    d.dims[:] = list(ba.dims)
    d.periodic[:] = [1, 1, 1]
    d.nu = sa.nu
    st = lib.lbm_create_domain(C.byref(d), C.byref(h))
    if st != lbm.LBM_OK:
        assert not alloc.live, "a failed creation leaked device buffers"
        return st
    u = np.ascontiguousarray(ba.u0, dtype=np.float32)
    c = np.ascontiguousarray(ba.c0, dtype=np.float32)
    note(lib.lbm_init_macro(h, 0, None, u.ctypes.data, c.ctypes.data, 0))
    note(lib.lbm_set_tape(h, 3))
    note(lib.lbm_step(h, 7))
    dldc = torch.ones(ba.flags.size, dtype=torch.float32, device="cuda")
    g = torch.empty(3 * ba.flags.size, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    note(lib.lbm_adjoint_step(h, 7, C.c_void_p(dldc.data_ptr()), None, C.c_void_p(g.data_ptr()), None))
    note(lib.lbm_sync(h))
    lib.lbm_destroy_domain(h)
    assert not alloc.live, f"{len(alloc.live)} device buffers leaked"
    return first


def test_every_failed_allocation_is_reported_and_nothing_leaks(lib):
    from paper_1807_02284_gb300 import lbm
    ref = FailingAllocator(fail_at=-1)
    assert _life_cycle(ref) == lbm.LBM_OK
    total = ref.count
    assert total > 10
    for k in range(total):
        a = FailingAllocator(fail_at=k)
        st = _life_cycle(a)
        assert st == lbm.LBM_ERR_OOM, f"allocation {k}: status {st}"
    torch.cuda.synchronize()


def test_domain_stays_usable_after_a_refused_block(lib):
    """A scale block whose allocation is refused leaves the domain exactly as it was: the
    next steps run and match a domain that never tried to add the block."""
    from paper_1807_02284_gb300 import lbm
    lib_ = lbm.load()
    sc = synth.random_scene(dims=(24, 20, 18), seed=21, periodic=(False, False, False),
                            spheres=[(12.0, 10.0, 9.0, 3.0)], inflow=(10, 9, 3.0, 0.08))
    b = sc.blocks[0]
    outs = []
    for refuse in (False, True):
        alloc = FailingAllocator(fail_at=-1)
        d = lbm.lbm_domain_desc()
        lib_.lbm_default_desc(C.byref(d))
        d.dims[:] = list(b.dims)
        d.nu = sc.nu
        d.cuda_stream = C.c_void_p(alloc.stream.cuda_stream)
        d.alloc = alloc.struct
        h = C.c_void_p()
        assert lib_.lbm_create_domain(C.byref(d), C.byref(h)) == lbm.LBM_OK
        fl = np.ascontiguousarray(b.flags, dtype=np.uint8)
        assert lib_.lbm_set_boundary(h, 0, lbm.LBM_BC_FLAGS, fl.ctypes.data, fl.nbytes, 0) == 0
        u = np.ascontiguousarray(b.u0, dtype=np.float32)
        assert lib_.lbm_init_macro(h, 0, None, u.ctypes.data, None, 0) == 0
        if refuse:
            alloc.fail_at = alloc.count + 4      # inside the new block's level buffers
            bid = C.c_int32()
            st = lib_.lbm_add_scale_block(h, (C.c_double * 3)(4.0, 4.0, 4.0), 0.5,
                                          (C.c_int32 * 3)(16, 16, 16), C.byref(bid))
            assert st == lbm.LBM_ERR_OOM
            info = lbm.lbm_block_info()
            assert lib_.lbm_get_block_info(h, 1, C.byref(info)) == lbm.LBM_ERR_INVALID_ARG
        assert lib_.lbm_step(h, 12) == lbm.LBM_OK
        f = np.empty(27 * b.flags.size, np.float32)
        assert lib_.lbm_read_field(h, 0, lbm.LBM_FIELD_F, lbm.LBM_F32, f.ctypes.data, f.nbytes, 0) == 0
        outs.append(f)
        lib_.lbm_destroy_domain(h)
        assert not alloc.live
    assert np.array_equal(outs[0], outs[1])
