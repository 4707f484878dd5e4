"""Python binding of the C-ABI in ``include/lbm.h`` (ctypes; argument marshalling only).

Every function of the header is exposed under the same name on the loaded library object
(``lib.lbm_step(...)``); :class:`Domain` is a thin convenience wrapper that converts numpy
arrays / torch tensors into pointers, raises :class:`LBMError` on a non-zero status and, by
default, routes the library's device allocations through PyTorch's caching allocator on the
current torch stream.  No solver arithmetic happens here: every step runs in the CUDA
library, and loading fails loudly if the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "liblbm.so")

# status codes
LBM_OK, LBM_ERR_INVALID_ARG, LBM_ERR_OOM, LBM_ERR_CUDA = 0, 1, 2, 3
LBM_ERR_DIVERGED, LBM_ERR_TIMEOUT, LBM_ERR_UNSUPPORTED, LBM_ERR_STATE = 4, 5, 6, 7
STATUS_NAMES = {0: "LBM_OK", 1: "LBM_ERR_INVALID_ARG", 2: "LBM_ERR_OOM", 3: "LBM_ERR_CUDA",
                4: "LBM_ERR_DIVERGED", 5: "LBM_ERR_TIMEOUT", 6: "LBM_ERR_UNSUPPORTED",
                7: "LBM_ERR_STATE"}
LBM_FP32, LBM_FP16_SHIFTED = 0, 1
LBM_BC_FLAGS, LBM_BC_INFLOW, LBM_BC_WALLS = 0, 1, 2
LBM_FIELD_F, LBM_FIELD_U, LBM_FIELD_SCALAR, LBM_FIELD_RHO, LBM_FIELD_FLAGS = 0, 1, 2, 3, 4
LBM_F32, LBM_F64, LBM_U8 = 0, 1, 2
LBM_MACRO_RHO, LBM_MACRO_U, LBM_MACRO_SCALAR = 0, 1, 2

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p)


class lbm_allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


class lbm_domain_desc(C.Structure):
    _fields_ = [("dims", C.c_int32 * 3), ("periodic", C.c_int32 * 3), ("nu", C.c_double),
                ("storage", C.c_int32), ("adaptive", C.c_int32), ("a", C.c_double),
                ("b", C.c_double), ("g_max", C.c_double), ("nu_hi", C.c_double * 4),
                ("c_src", C.c_double), ("cuda_stream", C.c_void_p), ("alloc", lbm_allocator),
                ("device", C.c_int32), ("grad_mode", C.c_int32)]

LBM_GRAD_LAGGED, LBM_GRAD_LOCAL = 0, 1


class lbm_block_info(C.Structure):
    _fields_ = [("dims", C.c_int32 * 3), ("origin", C.c_double * 3), ("h", C.c_double),
                ("nu", C.c_double), ("substeps", C.c_int32), ("steps", C.c_int64),
                ("tile", C.c_int32 * 2), ("ctas_per_sm", C.c_int32), ("parent", C.c_int32),
                ("nodes_per_thread", C.c_int32)]


INFLOW_RECORD = np.dtype([("x", "<i4"), ("y", "<i4"), ("z", "<i4"),
                          ("ux", "<f4"), ("uy", "<f4"), ("uz", "<f4")])

_P = C.c_void_p
_I = C.c_int32
_SIGNATURES = {
    "lbm_abi_version": (_I, []),
    "lbm_default_desc": (_I, [C.POINTER(lbm_domain_desc)]),
    "lbm_create_domain": (_I, [C.POINTER(lbm_domain_desc), C.POINTER(_P)]),
    "lbm_destroy_domain": (_I, [_P]),
    "lbm_add_scale_block": (_I, [_P, C.POINTER(C.c_double), C.c_double, C.POINTER(C.c_int32),
                                 C.POINTER(C.c_int32)]),
    "lbm_set_boundary": (_I, [_P, _I, _I, _P, C.c_size_t, _I]),
    "lbm_init_macro": (_I, [_P, _I, _P, _P, _P, _I]),
    "lbm_remove_scale_block": (_I, [_P, _I]),
    "lbm_detect_region": (_I, [_P, _I, C.c_double, C.c_double, C.POINTER(C.c_int64),
                               C.POINTER(C.c_int32)]),
    "lbm_init_block_from_parent": (_I, [_P, _I]),
    "lbm_build_dynamic_scale": (_I, [_P, _I, C.c_double, C.c_double, C.c_double, _I, _I,
                                     C.POINTER(C.c_int32)]),
    "lbm_build_static_scales": (_I, [_P, _I, C.c_double, C.c_double, C.c_double, _I,
                                     C.POINTER(C.c_int32)]),
    "lbm_build_static_scales_shadow": (_I, [_P, _I, C.c_double, C.c_double, C.c_double, _I, _I,
                                            C.POINTER(C.c_int32)]),
    "lbm_step": (_I, [_P, _I]),
    "lbm_sync": (_I, [_P]),
    "lbm_read_macro": (_I, [_P, _I, _I, _P, C.c_size_t, _I]),
    "lbm_read_field": (_I, [_P, _I, _I, _I, _P, C.c_size_t, _I]),
    "lbm_write_field": (_I, [_P, _I, _I, _I, _P, C.c_size_t, _I]),
    "lbm_reduce": (_I, [_P, _I, C.POINTER(C.c_double)]),
    "lbm_step_reduce": (_I, [_P, _I, C.POINTER(C.c_double)]),
    "lbm_step_reduce_async": (_I, [_P, _I, _P, C.POINTER(C.c_int64)]),
    "lbm_step_batch_reduce_async": (_I, [C.POINTER(_P), _I, _I, _P, C.POINTER(C.c_int64)]),
    "lbm_wait_results": (_I, [_P, C.c_int64]),
    "lbm_get_block_info": (_I, [_P, _I, C.POINTER(lbm_block_info)]),
    "lbm_step_batch": (_I, [C.POINTER(_P), _I, _I]),
    "lbm_step_batch_reduce": (_I, [C.POINTER(_P), _I, _I, C.POINTER(C.c_double)]),
    "lbm_plane_bytes": (C.c_size_t, [_P, _I]),
    "lbm_pack_plane": (_I, [_P, _I, _I, _P]),
    "lbm_unpack_plane": (_I, [_P, _I, _I, _P]),
    "lbm_step_slab": (_I, [_P, _I, _I, _P, _P, _P]),
    "lbm_step_phase": (_I, [_P, _I, _I, _I]),
    "lbm_mapping_boxes": (_I, [_P, _I, _I, _I, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "lbm_box_bytes": (C.c_size_t, [_P, _I, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "lbm_pack_box": (_I, [_P, _I, _I, C.POINTER(C.c_int32), C.POINTER(C.c_int32), _P]),
    "lbm_unpack_box": (_I, [_P, _I, _I, C.POINTER(C.c_int32), C.POINTER(C.c_int32), _P, _I]),
    "lbm_reduce_batch": (_I, [C.POINTER(_P), _I, _I, C.POINTER(C.c_double)]),
    "lbm_set_inflow_batch": (_I, [C.POINTER(_P), _I, C.POINTER(_P), C.POINTER(C.c_int32)]),
    "lbm_set_tape": (_I, [_P, _I]),
    "lbm_adjoint_step": (_I, [_P, _I, _P, _P, _P, _P]),
    "lbm_adjoint_block_grad": (_I, [_P, _I, _P]),
    "lbm_reduce_noalloc": (_I, [_P, _I, _P, C.c_int64, _P, _P]),
    "lbm_barrier_selftest": (_I, [_I, C.c_double, _P]),
    "lbm_last_error": (C.c_char_p, [_P]),
}
LBM_REDUCE_NOALLOC_MAX_NODES = 67108864
LBM_PHASE_BEGIN, LBM_PHASE_REFERENCE, LBM_PHASE_BLOCK, LBM_PHASE_POST, LBM_PHASE_END = 0, 1, 2, 3, 4
LBM_BOX_PRIOR_SOURCE, LBM_BOX_POST_TARGET = 0, 1
LBM_LEVEL_CURRENT, LBM_LEVEL_START = 0, 1

_lib = None
ABI_VERSION = 5      # lbm_abi_version() of the include/lbm.h these structs mirror


def load(path: str = LIB_PATH):
    """Loads the built CUDA library (raises if it has not been built, or was built from
    another version of the ABI than the structs declared here)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing "
                           "(run __graft_entry__.build() or python -m paper_1807_02284_gb300.build)")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if lib.lbm_abi_version() != ABI_VERSION:
        raise RuntimeError(f"{path} has ABI version {lib.lbm_abi_version()}, the binding "
                           f"expects {ABI_VERSION}: rebuild the library")
    _lib = lib
    return lib


class LBMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _ptr(a):
    """Pointer and on-device flag of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data, 0
    import torch
    if isinstance(a, torch.Tensor):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), 1 if a.is_cuda else 0
    raise TypeError(f"unsupported array type {type(a)}")


def _nbytes(a):
    if isinstance(a, np.ndarray):
        return a.nbytes
    return a.numel() * a.element_size()


class Domain:
    """Owning wrapper of one ``lbm_domain`` handle."""

    def __init__(self, dims: Sequence[int], nu: float, periodic=(False, False, False),
                 storage: str = "fp32", adaptive: bool = True, a: float = -4.0, b: float = 5.0,
                 g_max: float = 0.1, nu_hi=(0.005, 0.007, 0.009, 0.01), c_src: float = 1.0,
                 stream=None, torch_allocator: bool = True, device: int = 0,
                 grad_mode: str = "lagged"):
        self.lib = load()
        self.handle = C.c_void_p()
        d = lbm_domain_desc()
        self.lib.lbm_default_desc(C.byref(d))
        d.dims[:] = [int(v) for v in dims]
        d.periodic[:] = [1 if p else 0 for p in periodic]
        d.nu = float(nu)
        d.storage = LBM_FP16_SHIFTED if storage in ("fp16", "fp16s", LBM_FP16_SHIFTED) else LBM_FP32
        d.adaptive = 1 if adaptive else 0
        d.a, d.b, d.g_max = float(a), float(b), float(g_max)
        d.nu_hi[:] = [float(v) for v in nu_hi]
        d.c_src = float(c_src)
        d.device = int(device)
        d.grad_mode = LBM_GRAD_LOCAL if grad_mode == "local" else LBM_GRAD_LAGGED
        self._keep = []
        if stream is None:
            import torch
            stream = torch.cuda.current_stream(device)
            if stream.cuda_stream == 0:
                # the default stream has no handle to pass (NULL would make the library create
                # a private stream torch does not know): give the domain a stream of its own
                # that torch_stream names, so that waits on torch_stream order its work
                stream = torch.cuda.Stream(device=device)
        self.torch_stream = stream
        d.cuda_stream = C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else stream)
        if torch_allocator:
            import torch

            dev = int(device)
            tstream = stream

            def _alloc(nbytes, ctx):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, tstream)
                except Exception:  # OOM or other failure -> NULL (library reports LBM_ERR_OOM)
                    return None

            def _free(p, nbytes, ctx):
                torch.cuda.caching_allocator_delete(p)

            fa, ff = ALLOC_FN(_alloc), FREE_FN(_free)
            self._keep += [fa, ff]
            d.alloc = lbm_allocator(fa, ff, None)
        self.desc = d
        self.storage = d.storage
        self.check(self.lib.lbm_create_domain(C.byref(d), C.byref(self.handle)), create=True)

    # -------------------------------------------------------------------------- plumbing
    def check(self, st, create=False):
        if st != LBM_OK:
            h = None if create else self.handle
            msg = self.lib.lbm_last_error(h)
            raise LBMError(st, msg.decode() if msg else "")
        return st

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            self.lib.lbm_destroy_domain(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------------------- API
    def add_scale_block(self, origin, h, dims) -> int:
        o = (C.c_double * 3)(*[float(v) for v in origin])
        dd = (C.c_int32 * 3)(*[int(v) for v in dims])
        bid = C.c_int32()
        self.check(self.lib.lbm_add_scale_block(self.handle, o, float(h), dd, C.byref(bid)))
        return bid.value

    def remove_scale_block(self, block: int):
        self.check(self.lib.lbm_remove_scale_block(self.handle, int(block)))

    def detect_region(self, g_threshold: float, u_threshold: float, block: int = 0):
        """(count, box) with box = (x0, y0, z0, x1, y1, z1), or (0, None)."""
        n = C.c_int64()
        box = (C.c_int32 * 6)()
        self.check(self.lib.lbm_detect_region(self.handle, int(block), float(g_threshold),
                                              float(u_threshold), C.byref(n), box))
        return (int(n.value), tuple(box)) if n.value else (0, None)

    def init_block_from_parent(self, block: int):
        self.check(self.lib.lbm_init_block_from_parent(self.handle, int(block)))

    def build_dynamic_scale(self, h: float, g_threshold: float, u_threshold: float,
                            margin: int = 2, replace_last: bool = False, src_block: int = 0) -> int:
        bid = C.c_int32()
        self.check(self.lib.lbm_build_dynamic_scale(self.handle, int(src_block), float(h),
                                                    float(g_threshold), float(u_threshold),
                                                    int(margin), 1 if replace_last else 0,
                                                    C.byref(bid)))
        return bid.value

    def build_static_scales(self, n_scales: int, h_min: float, d_max: float, wake: float = 0.0,
                            flow_axis: int = 0) -> int:
        n = C.c_int32()
        self.check(self.lib.lbm_build_static_scales(self.handle, int(n_scales), float(h_min),
                                                    float(d_max), float(wake), int(flow_axis),
                                                    C.byref(n)))
        return n.value

    def build_static_scales_shadow(self, n_scales: int, h_min: float, d_max: float,
                                   wake: float, flow_axis: int = 0, n_light: int = 16) -> int:
        """Static scales whose wakes follow the soft shadow of the obstacles lit by the inlet."""
        n = C.c_int32()
        self.check(self.lib.lbm_build_static_scales_shadow(self.handle, int(n_scales), float(h_min),
                                                           float(d_max), float(wake), int(flow_axis),
                                                           int(n_light), C.byref(n)))
        return n.value

    def info(self, block=0) -> lbm_block_info:
        i = lbm_block_info()
        self.check(self.lib.lbm_get_block_info(self.handle, block, C.byref(i)))
        return i

    def n_blocks(self) -> int:
        """Number of blocks of the domain (the reference block, refined and far-field ones)."""
        i, n = lbm_block_info(), 0
        while self.lib.lbm_get_block_info(self.handle, n, C.byref(i)) == LBM_OK:
            n += 1
        return n

    def n_nodes(self, block=0) -> int:
        i = self.info(block)
        return int(i.dims[0]) * int(i.dims[1]) * int(i.dims[2])

    def set_flags(self, flags, block=0):
        if isinstance(flags, np.ndarray):
            flags = np.ascontiguousarray(flags, dtype=np.uint8)
        p, dev = _ptr(flags)
        self.check(self.lib.lbm_set_boundary(self.handle, block, LBM_BC_FLAGS, p, _nbytes(flags), dev))

    def set_walls(self, faces, obstacles=False):
        """No-slip wall faces of block 0: six booleans (x-, x+, y-, y+, z-, z+); with
        ``obstacles`` the surface voxels of the obstacles are walls too, in every block."""
        m = np.ascontiguousarray([1 if f else 0 for f in faces] + [1 if obstacles else 0],
                                 dtype=np.uint8)
        self.check(self.lib.lbm_set_boundary(self.handle, 0, LBM_BC_WALLS, m.ctypes.data, 7, 0))

    def set_inflow(self, records, block=0):
        if isinstance(records, np.ndarray):
            records = np.ascontiguousarray(records, dtype=INFLOW_RECORD)
        p, dev = _ptr(records)
        self.check(self.lib.lbm_set_boundary(self.handle, block, LBM_BC_INFLOW, p, _nbytes(records), dev))

    def init_macro(self, u, rho=None, c=None, block=0):
        arrs = []
        for a in (rho, u, c):
            if isinstance(a, np.ndarray):
                a = np.ascontiguousarray(a, dtype=np.float32)
            arrs.append(a)
        rho, u, c = arrs
        devs = {_ptr(a)[1] for a in (rho, u, c) if a is not None}
        if len(devs) != 1:
            raise ValueError("rho, u and c must all live on the host or all on the device")
        self.check(self.lib.lbm_init_macro(self.handle, block, _ptr(rho)[0], _ptr(u)[0],
                                           _ptr(c)[0], devs.pop()))

    def step(self, n=1):
        self.check(self.lib.lbm_step(self.handle, int(n)))

    def sync(self):
        self.check(self.lib.lbm_sync(self.handle))

    def read_field(self, field, dtype=LBM_F64, block=0, out=None):
        N = self.n_nodes(block)
        count = {LBM_FIELD_F: 27 * N, LBM_FIELD_U: 3 * N, LBM_FIELD_SCALAR: N,
                 LBM_FIELD_RHO: N, LBM_FIELD_FLAGS: N}[field]
        npdt = {LBM_F32: np.float32, LBM_F64: np.float64, LBM_U8: np.uint8}[dtype]
        if out is None:
            out = np.empty(count, dtype=npdt)
        p, dev = _ptr(out)
        self.check(self.lib.lbm_read_field(self.handle, block, field, dtype, p, _nbytes(out), dev))
        return out

    def write_field(self, field, data, block=0):
        if isinstance(data, np.ndarray):
            if data.dtype not in (np.float32, np.float64):
                data = data.astype(np.float64)
            data = np.ascontiguousarray(data)
            dtype = LBM_F64 if data.dtype == np.float64 else LBM_F32
        else:
            import torch
            dtype = LBM_F64 if data.dtype == torch.float64 else LBM_F32
        p, dev = _ptr(data)
        self.check(self.lib.lbm_write_field(self.handle, block, field, dtype, p, _nbytes(data), dev))

    def reduce(self, block=0) -> np.ndarray:
        out = (C.c_double * 5)()
        self.check(self.lib.lbm_reduce(self.handle, block, out))
        return np.array(list(out))

    def plane_bytes(self, direction=0) -> int:
        """Bytes of a packed z-plane: direction +1 / -1 carry the 9 populations with c_z = +1 / -1,
        direction 0 all 27 (plus velocity, scalar and flags)."""
        return int(self.lib.lbm_plane_bytes(self.handle, int(direction)))

    def _plane_buffer(self, buf, direction):
        p, dev = _ptr(buf)
        if not dev:
            raise ValueError("plane buffers are device memory")
        if _nbytes(buf) < self.plane_bytes(direction) or (p or 0) % 16:
            raise ValueError("a plane buffer holds plane_bytes(direction) bytes, 16-byte aligned")
        return p

    def pack_plane(self, z, buf, direction=0):
        """Copies z-plane `z` of the current state into the device tensor `buf`."""
        self.check(self.lib.lbm_pack_plane(self.handle, int(z), int(direction),
                                           self._plane_buffer(buf, direction)))

    def unpack_plane(self, z, buf, direction=0):
        """Copies the device tensor `buf` into z-plane `z` of the current state."""
        self.check(self.lib.lbm_unpack_plane(self.handle, int(z), int(direction),
                                             self._plane_buffer(buf, direction)))

    def step_slab(self, lo, hi, send_lo=None, send_hi=None, pack_stream=None):
        """``lbm_step_slab``: one step of a slab, its send planes stepped first and packed on
        ``pack_stream`` (a torch stream, or None for an internal one) while the other owned
        planes step; halo planes are left to the next unpack."""
        plo = self._plane_buffer(send_lo, -1) if lo else None
        phi = self._plane_buffer(send_hi, +1) if hi else None
        ps = None if pack_stream is None else C.c_void_p(
            pack_stream.cuda_stream if hasattr(pack_stream, "cuda_stream") else pack_stream)
        self.check(self.lib.lbm_step_slab(self.handle, 1 if lo else 0, 1 if hi else 0, plo, phi, ps))

    def step_phase(self, phase, block=0, compute=True):
        """One phase of a reference step (LBM_PHASE_*), computed or only advancing levels."""
        self.check(self.lib.lbm_step_phase(self.handle, int(phase), int(block), int(bool(compute))))

    def mapping_boxes(self, block, kind, other):
        """Node boxes [(lo, hi), ...] of block `other` exchanged by refined block `block`'s
        mappings (LBM_BOX_PRIOR_SOURCE: its source, six faces; LBM_BOX_POST_TARGET: what its
        post-mapping writes into `other`)."""
        buf = (C.c_int32 * 36)()
        n = C.c_int32(0)
        self.check(self.lib.lbm_mapping_boxes(self.handle, int(block), int(kind), int(other),
                                              buf, C.byref(n)))
        return [(tuple(buf[6 * i:6 * i + 3]), tuple(buf[6 * i + 3:6 * i + 6]))
                for i in range(n.value)]

    @staticmethod
    def _box(lo, hi):
        return (C.c_int32 * 3)(*[int(v) for v in lo]), (C.c_int32 * 3)(*[int(v) for v in hi])

    def box_bytes(self, block, lo, hi) -> int:
        l, h = self._box(lo, hi)
        return int(self.lib.lbm_box_bytes(self.handle, int(block), l, h))

    def _box_buffer(self, buf, block, lo, hi):
        p, dev = _ptr(buf)
        if not dev:
            raise ValueError("box buffers are device memory")
        if _nbytes(buf) < self.box_bytes(block, lo, hi) or (p or 0) % 16:
            raise ValueError("a box buffer holds box_bytes() bytes, 16-byte aligned")
        return p

    def pack_box(self, block, level, lo, hi, buf):
        """Copies a node box of block `block` (level LBM_LEVEL_*) into the device tensor buf."""
        l, h = self._box(lo, hi)
        self.check(self.lib.lbm_pack_box(self.handle, int(block), int(level), l, h,
                                         self._box_buffer(buf, block, lo, hi)))

    def unpack_box(self, block, level, lo, hi, buf, skip_flags=0):
        """Copies the device tensor buf into a node box, leaving nodes with skip_flags bits."""
        l, h = self._box(lo, hi)
        self.check(self.lib.lbm_unpack_box(self.handle, int(block), int(level), l, h,
                                           self._box_buffer(buf, block, lo, hi), int(skip_flags)))

    def step_reduce(self, n=1) -> np.ndarray:
        """``lbm_step_reduce``: n steps, then block 0's diagnostics (mass, momentum x/y/z,
        kinetic energy), summed by the last step's own kernel where the domain allows."""
        out = (C.c_double * 5)()
        self.check(self.lib.lbm_step_reduce(self.handle, int(n), out))
        return np.array(list(out))

    def step_reduce_async(self, n, out) -> int:
        """``lbm_step_reduce_async``: enqueues n steps and block 0's diagnostics, to be copied
        into ``out`` (5 float64 values in host memory, pinned for an asynchronous copy: a
        numpy array or a CPU torch tensor); returns the ticket for ``wait_results``."""
        ptr, dev = _ptr(out)
        if dev or _nbytes(out) < 5 * 8 or str(out.dtype) not in ("float64", "torch.float64"):
            raise ValueError("out must be 5 float64 values in host memory")
        t = C.c_int64()
        self.check(self.lib.lbm_step_reduce_async(self.handle, int(n), C.c_void_p(ptr), C.byref(t)))
        return t.value

    def wait_results(self, ticket: int):
        self.check(self.lib.lbm_wait_results(self.handle, int(ticket)))

    def set_tape(self, every):
        self.check(self.lib.lbm_set_tape(self.handle, int(every)))

    def adjoint_step(self, n_steps, dL_dc, dL_du0, dL_du=None, dL_dinflow=None):
        pc, _ = _ptr(dL_dc)
        pu, _ = _ptr(dL_du)
        p0, _ = _ptr(dL_du0)
        pi, _ = _ptr(dL_dinflow)
        self.check(self.lib.lbm_adjoint_step(self.handle, int(n_steps), pc, pu, p0, pi))

    def adjoint_block_grad(self, block, out):
        p, _ = _ptr(out)
        self.check(self.lib.lbm_adjoint_block_grad(self.handle, int(block), p))


def step_batch(domains: Sequence[Domain], steps: int):
    """``lbm_step_batch`` over the handles of several domains."""
    lib = load()
    arr = (C.c_void_p * len(domains))(*[d.handle.value for d in domains])
    st = lib.lbm_step_batch(arr, len(domains), int(steps))
    if st != LBM_OK:
        domains[0].check(st)


def step_batch_reduce(domains: Sequence[Domain], steps: int) -> np.ndarray:
    """``lbm_step_batch_reduce``: the batched steps, then every member's five diagnostics
    (shape (n, 5)) summed by the last step's own kernel."""
    lib = load()
    arr = (C.c_void_p * len(domains))(*[d.handle.value for d in domains])
    out = (C.c_double * (5 * len(domains)))()
    st = lib.lbm_step_batch_reduce(arr, len(domains), int(steps), out)
    if st != LBM_OK:
        domains[0].check(st)
    return np.array(list(out)).reshape(len(domains), 5)


def step_batch_reduce_async(domains: Sequence[Domain], steps: int, out) -> int:
    """``lbm_step_batch_reduce_async``: the batched steps and every member's diagnostics,
    copied into ``out`` (5 n float64 values in host memory, pinned for an asynchronous copy);
    returns the ticket to pass to ``domains[0].wait_results``."""
    lib = load()
    ptr, dev = _ptr(out)
    if dev or _nbytes(out) < 5 * 8 * len(domains) or str(out.dtype) not in ("float64", "torch.float64"):
        raise ValueError("out must be 5 n float64 values in host memory")
    arr = (C.c_void_p * len(domains))(*[d.handle.value for d in domains])
    t = C.c_int64()
    st = lib.lbm_step_batch_reduce_async(arr, len(domains), int(steps), C.c_void_p(ptr), C.byref(t))
    if st != LBM_OK:
        domains[0].check(st)
    return t.value


def set_inflow_batch(domains: Sequence[Domain], records: Sequence[np.ndarray]):
    """``lbm_set_inflow_batch``: inflow records (host arrays of INFLOW_RECORD) for block 0
    of every domain, staged and applied together."""
    lib = load()
    n = len(domains)
    recs = [np.ascontiguousarray(r, dtype=INFLOW_RECORD) for r in records]
    arr = (C.c_void_p * n)(*[d.handle.value for d in domains])
    ptrs = (C.c_void_p * n)(*[r.ctypes.data if r.size else None for r in recs])
    counts = (C.c_int32 * n)(*[int(r.size) for r in recs])
    st = lib.lbm_set_inflow_batch(arr, n, ptrs, counts)
    if st != LBM_OK:
        domains[0].check(st)


def reduce_batch(domains: Sequence[Domain], block: int = 0) -> np.ndarray:
    """``lbm_reduce_batch``: the five diagnostics of every domain, shape (n, 5)."""
    lib = load()
    arr = (C.c_void_p * len(domains))(*[d.handle.value for d in domains])
    out = (C.c_double * (5 * len(domains)))()
    st = lib.lbm_reduce_batch(arr, len(domains), int(block), out)
    if st != LBM_OK:
        domains[0].check(st)
    return np.array(list(out)).reshape(len(domains), 5)
