"""GPU parity of the no-slip wall faces (Sec. 6.1 second-order wall, regularized on-node
reading) against the FP64 oracle through the C-ABI: walls on faces, edges and corners,
with obstacles and an inflow disk in the block."""
import dataclasses

import numpy as np
import pytest

import synth
from oracle import grid
from tests.helpers import gpu_domain, gpu_state, max_err, oracle_params, oracle_state

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("walls", [(False, False, False, False, True, True),    # floor + lid
                                   (False, True, True, False, True, False),     # edges, corner
                                   (False, True, True, True, True, True)])      # five walls
def test_wall_faces_match_oracle(lib, walls):
    sc = synth.random_scene(dims=(26, 22, 18), seed=51, periodic=(False, False, False),
                            spheres=[(13.0, 11.0, 9.0, 3.0)], inflow=(11, 9, 3.0, 0.07), nu=0.01)
    b = sc.blocks[0]
    dom = gpu_domain(sc)
    dom.set_walls(walls)
    st = oracle_state(sc)
    p = dataclasses.replace(oracle_params(sc), walls=walls)
    for _ in range(8):
        dom.step(1)
        st = grid.step(st, p)
    f, u, c = gpu_state(dom, b.shape_zyx)
    umax = float(np.abs(st.u.numpy()).max())
    eu, ef, ec = max_err(u, st.u.numpy()), max_err(f, st.f.numpy()), max_err(c, st.c.numpy())
    print(f"walls {walls}: |du|={eu:.2e} (max|u| {umax:.3f}) |df|={ef:.2e} |dc|={ec:.2e}")
    assert eu <= 1e-5 * umax and ef <= 2e-7 and ec <= 1e-6
    # wall nodes (not inflow, not obstacle) are at rest
    z = np.zeros(b.shape_zyx, bool)
    if walls[4]:
        z[0] = True
    if walls[5]:
        z[-1] = True
    keep = z & ((b.flags & 3) == 0)
    assert np.abs(u[:, keep]).max() < 1e-7
    dom.close()


def test_wall_argument_checks(lib):
    from paper_1807_02284_gb300 import lbm
    dom = lbm.Domain((12, 12, 12), 0.01, periodic=(True, False, False))
    with pytest.raises(lbm.LBMError) as ei:
        dom.set_walls((True, False, False, False, False, False))   # x is periodic
    assert ei.value.status == lbm.LBM_ERR_INVALID_ARG
    dom.set_walls((False, False, False, False, True, True))
    with pytest.raises(lbm.LBMError) as ei:
        dom.set_tape(2)
    assert ei.value.status == lbm.LBM_ERR_UNSUPPORTED
    dom.set_walls((False,) * 6)
    dom.step(2)
    dom.sync()
    dom.close()
