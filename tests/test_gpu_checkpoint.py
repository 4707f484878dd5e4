"""Checkpoint and resume through the C-ABI: the state read back with lbm_read_field
(populations, stored velocity, scalar) and written into a fresh domain continues
bit-identically, for FP32 and FP16-shifted storage."""
import numpy as np
import pytest

import synth
from tests.helpers import gpu_domain

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_resume_from_saved_state_is_bit_identical(lib, storage):
    from paper_1807_02284_gb300 import lbm
    sc = synth.random_scene(dims=(30, 26, 22), seed=14, periodic=(False, True, True),
                            spheres=[(15.0, 13.0, 11.0, 4.0)], inflow=(13, 11, 4.0, 0.1))
    a = gpu_domain(sc, storage)
    a.step(10)
    saved = {f: a.read_field(f, lbm.LBM_F64) for f in (lbm.LBM_FIELD_F, lbm.LBM_FIELD_U,
                                                        lbm.LBM_FIELD_SCALAR)}
    a.step(10)
    b = gpu_domain(sc, storage)                  # same flags, fresh state
    for f, arr in saved.items():
        b.write_field(f, arr)
    b.step(10)
    for f in (lbm.LBM_FIELD_F, lbm.LBM_FIELD_U, lbm.LBM_FIELD_SCALAR):
        assert np.array_equal(a.read_field(f, lbm.LBM_F32), b.read_field(f, lbm.LBM_F32))
    a.close()
    b.close()
