"""A host stand-in for ``lbm.Domain`` in the block-placement tests: the FP64 oracle's
continuous-scale domain (``oracle.coupling.MultiScale``) behind the interface that
``sharding.PlacedDomain`` uses (phases, mapping boxes, node-box packing), so that the
placement's exchange plan and transport run on CPU ranks without a GPU.  Boxes follow the
library's geometry (the six faces of a block's scale boundary in its source, the interior
span of a block in a coarser one); a packed box holds the 27 populations, the velocity and
the scalar of every box node in float64."""
import math
import types

import numpy as np
import torch

from oracle import coupling, grid
from paper_1807_02284_gb300 import lbm


class OraclePlacedDomain:
    box_device = "cpu"

    def __init__(self, scene):
        self.ms = coupling.MultiScale.build(scene)
        self.ms.saved = None

    # ------------------------------------------------------------------ structure
    def n_blocks(self):
        return len(self.ms.blocks)

    def info(self, b):
        blk = self.ms.blocks[b]
        return types.SimpleNamespace(parent=(-1 if b == 0 or blk.far else blk.parent))

    def mapping_boxes(self, b, kind, other):
        B, O = self.ms.blocks[b], self.ms.blocks[other]
        nB, nO = np.array(B.dims), np.array(O.dims)
        if kind == lbm.LBM_BOX_PRIOR_SOURCE:
            assert other == B.parent
            out = []
            for f in range(6):
                lo, hi = [0] * 3, [0] * 3
                for a in range(3):
                    p0, p1 = B.origin[a], B.origin[a] + (nB[a] - 1) * B.h
                    if a == f // 2:
                        p0 = p1 = p1 if f % 2 else p0
                    i0 = min(max(math.floor((p0 - O.origin[a]) / O.h), 0), max(nO[a] - 2, 0))
                    i1 = min(max(math.floor((p1 - O.origin[a]) / O.h), 0), max(nO[a] - 2, 0))
                    lo[a], hi[a] = i0, min(i1 + 1, nO[a] - 1)
                out.append((tuple(lo), tuple(hi)))
            return out
        if not (O.h > B.h and not O.far):
            return []
        lo, hi = B.interior_lo_hi()
        blo = [max(0, math.ceil((lo[a] - 1e-9 - O.origin[a]) / O.h)) for a in range(3)]
        bhi = [min(nO[a] - 1, math.floor((hi[a] + 1e-9 - O.origin[a]) / O.h)) for a in range(3)]
        if any(blo[a] > bhi[a] for a in range(3)):
            return []
        return [(tuple(blo), tuple(bhi))]

    # ------------------------------------------------------------------ node boxes
    @staticmethod
    def box_bytes(b, lo, hi):
        n = int(np.prod([hi[a] - lo[a] + 1 for a in range(3)]))
        return n * 31 * 8

    def _state(self, b, level):
        return self.ms.saved[b] if level == lbm.LBM_LEVEL_START else self.ms.blocks[b].state

    def _set_state(self, b, level, st):
        if level == lbm.LBM_LEVEL_START:
            self.ms.saved[b] = st
        else:
            self.ms.blocks[b].state = st

    @staticmethod
    def _sl(lo, hi):
        return (slice(lo[2], hi[2] + 1), slice(lo[1], hi[1] + 1), slice(lo[0], hi[0] + 1))

    def pack_box(self, b, level, lo, hi, buf):
        st = self._state(b, level)
        z, y, x = self._sl(lo, hi)
        parts = [st.f[:, z, y, x].reshape(27, -1), st.u[:, z, y, x].reshape(3, -1),
                 st.c[z, y, x].reshape(1, -1)]
        buf.view(torch.float64).copy_(torch.cat(parts).reshape(-1))

    def unpack_box(self, b, level, lo, hi, buf, skip=0):
        st = self._state(b, level).clone()
        z, y, x = self._sl(lo, hi)
        v = buf.view(torch.float64).reshape(31, -1)
        shape = st.c[z, y, x].shape
        keep = ((st.flags[z, y, x] & skip) != 0)
        f = st.f[:, z, y, x]
        u = st.u[:, z, y, x]
        c = st.c[z, y, x]
        st.f[:, z, y, x] = torch.where(keep[None], f, v[:27].reshape((27,) + shape))
        st.u[:, z, y, x] = torch.where(keep[None], u, v[27:30].reshape((3,) + shape))
        st.c[z, y, x] = torch.where(keep, c, v[30].reshape(shape))
        self._set_state(b, level, st)

    # ------------------------------------------------------------------ phases
    def step_phase(self, phase, block=0, compute=True):
        ms = self.ms
        if phase == lbm.LBM_PHASE_BEGIN:
            ms.begin()
        elif phase == lbm.LBM_PHASE_REFERENCE:
            if compute:
                ms.step_reference()
        elif phase == lbm.LBM_PHASE_BLOCK:
            if compute:
                ms.step_block(block)
        elif phase == lbm.LBM_PHASE_POST:
            if compute:
                ms.post_block(block)
        elif phase == lbm.LBM_PHASE_END:
            ms.end()

    def sync(self):
        pass
