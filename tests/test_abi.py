"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads, exports every entry
point declared in include/lbm.h, and rejects bad arguments on the host before touching a
GPU."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    from paper_1807_02284_gb300 import build
    return build.build()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(lbm_[a-z0-9_]+)\s*\(",
                             text, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_hot_path_entry_points():
    names = _declared()
    for n in ("lbm_create_domain", "lbm_destroy_domain", "lbm_add_scale_block",
              "lbm_set_boundary", "lbm_init_macro", "lbm_step", "lbm_read_macro",
              "lbm_step_batch", "lbm_set_tape", "lbm_adjoint_step", "lbm_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(built):
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True,
                         check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    missing = _declared() - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"


def test_library_loads_and_validates_on_host(built):
    from paper_1807_02284_gb300 import lbm
    lib = lbm.load()
    assert lib.lbm_abi_version() == 5
    d = lbm.lbm_domain_desc()
    assert lib.lbm_default_desc(C.byref(d)) == lbm.LBM_OK
    assert (d.a, d.b, d.g_max) == (-4.0, 5.0, 0.1)
    assert list(d.nu_hi) == [0.005, 0.007, 0.009, 0.01]
    assert d.adaptive == 1 and d.storage == lbm.LBM_FP32
    h = C.c_void_p()
    # dims not filled in -> rejected before any CUDA call
    assert lib.lbm_create_domain(C.byref(d), C.byref(h)) == lbm.LBM_ERR_INVALID_ARG
    assert b"dims" in lib.lbm_last_error(None)
    d.dims[:] = [8, 8, 8]
    d.nu = -1.0
    assert lib.lbm_create_domain(C.byref(d), C.byref(h)) == lbm.LBM_ERR_INVALID_ARG
    d.nu = 0.01
    d.storage = 7
    assert lib.lbm_create_domain(C.byref(d), C.byref(h)) == lbm.LBM_ERR_INVALID_ARG
    assert lib.lbm_create_domain(None, C.byref(h)) == lbm.LBM_ERR_INVALID_ARG
    # null handles
    assert lib.lbm_step(None, 1) == lbm.LBM_ERR_INVALID_ARG
    assert lib.lbm_sync(None) == lbm.LBM_ERR_INVALID_ARG
    assert lib.lbm_destroy_domain(None) == lbm.LBM_OK
    assert lib.lbm_step_reduce(None, 1, None) == lbm.LBM_ERR_INVALID_ARG
    assert lib.lbm_step_reduce_async(None, 1, None, None) == lbm.LBM_ERR_INVALID_ARG
    assert lib.lbm_wait_results(None, 1) == lbm.LBM_ERR_INVALID_ARG
    assert lib.lbm_set_tape(None, 1) == lbm.LBM_ERR_INVALID_ARG
    assert lib.lbm_adjoint_step(None, 1, None, None, None, None) == lbm.LBM_ERR_INVALID_ARG
    assert lib.lbm_reduce_batch(None, 0, 0, None) == lbm.LBM_ERR_INVALID_ARG
    assert lib.lbm_set_inflow_batch(None, 0, None, None) == lbm.LBM_ERR_INVALID_ARG
    assert lib.lbm_step_batch_reduce(None, 1, 1, None) == lbm.LBM_ERR_INVALID_ARG
    assert lib.lbm_step_batch_reduce_async(None, 1, 1, None, None) == lbm.LBM_ERR_INVALID_ARG
    assert lib.lbm_plane_bytes(None, 0) == 0
    assert lib.lbm_step_slab(None, 1, 1, None, None, None) == lbm.LBM_ERR_INVALID_ARG
    for fn in (lib.lbm_pack_plane, lib.lbm_unpack_plane):
        assert fn(None, 0, 0, None) == lbm.LBM_ERR_INVALID_ARG
    assert lib.lbm_step_phase(None, 0, 0, 1) == lbm.LBM_ERR_INVALID_ARG
    assert lib.lbm_mapping_boxes(None, 1, 0, 0, None, None) == lbm.LBM_ERR_INVALID_ARG
    assert lib.lbm_box_bytes(None, 0, None, None) == 0
    assert lib.lbm_pack_box(None, 0, 0, None, None, None) == lbm.LBM_ERR_INVALID_ARG
    assert lib.lbm_unpack_box(None, 0, 0, None, None, None, 0) == lbm.LBM_ERR_INVALID_ARG


def test_struct_layouts_match_header():
    from paper_1807_02284_gb300 import lbm
    # int32[3] int32[3] double int32 int32 double*3 double[4] double void* {3 ptr} int32 (+pad)
    assert C.sizeof(lbm.lbm_domain_desc) == 12 + 12 + 8 + 4 + 4 + 24 + 32 + 8 + 8 + 24 + 8
    assert lbm.INFLOW_RECORD.itemsize == 24
