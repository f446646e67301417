"""ctypes declarations of the C ABI in ``include/rd.h`` (argument
marshalling only).  Loading fails loudly when the library is not built."""
from __future__ import annotations

import ctypes
import os

from . import build as _build

MAX_S = 4

RD_OK, RD_EINVAL, RD_ENOMEM, RD_ECUDA, RD_EUNSTABLE, RD_ENONFINITE, RD_ETIMEOUT, \
    RD_EBUDGET, RD_EUNSUPPORTED, RD_EBOUNDS = range(10)
BC = {"neumann": 0, "periodic": 1, "dirichlet": 2}
MODEL = {"diffusion": 0, "brusselator": 1, "ch_front": 2, "air": 3, "turing": 4,
         "ch_table1": 5}
STORAGE = {"f32": 0, "bf16": 1}
WIND = {None: 0, "log": 1, "const": 2, "3d": 3}
KERNEL = {"march": 0, "shared": 1, "tiles": 2, "resident": 3}
FLAG_NO_ALLOC, FLAG_FORCE = 1, 2


class RdConfig(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("nspecies", ctypes.c_int32), ("model", ctypes.c_int32), ("storage", ctypes.c_int32),
        ("h", ctypes.c_double), ("dt", ctypes.c_double),
        ("D", (ctypes.c_double * 3) * MAX_S),
        ("bc", (ctypes.c_int32 * 6) * MAX_S),
        ("bc_value", (ctypes.c_double * 6) * MAX_S),
        ("params", ctypes.c_double * 8),
        ("wind_kind", ctypes.c_int32), ("stencil", ctypes.c_int32),
        ("wind_u0", ctypes.c_double),
        ("src_x", ctypes.c_int32), ("src_y", ctypes.c_int32), ("src_z", ctypes.c_int32),
        ("src_species", ctypes.c_int32), ("src_rate", ctypes.c_double),
        ("flags", ctypes.c_int32), ("reserved1", ctypes.c_int32),
        ("wind_vel", ctypes.c_double * 3), ("wind_tau", ctypes.c_double),
    ]


class RdTuning(ctypes.Structure):
    _fields_ = [("tsteps", ctypes.c_int32), ("tile_q", ctypes.c_int32),
                ("tile_y", ctypes.c_int32), ("zchunk", ctypes.c_int32),
                ("graph", ctypes.c_int32), ("regcap", ctypes.c_int32)]

    def as_dict(self):
        return dict(tsteps=self.tsteps, tile_q=self.tile_q, tile_y=self.tile_y,
                    zchunk=self.zchunk, graph=self.graph, regcap=self.regcap)


_P = ctypes.c_void_p
_I = ctypes.c_int
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_SZ = ctypes.c_size_t
_CFG = ctypes.POINTER(RdConfig)
_TUN = ctypes.POINTER(RdTuning)
_PP = ctypes.POINTER(ctypes.c_void_p)
_DP = ctypes.POINTER(ctypes.c_double)

# name -> (restype, argtypes); every symbol include/rd.h declares
SIGNATURES = {
    "rd_config_init": (_I, [_CFG]),
    "rd_query_sizes": (_I, [_CFG, ctypes.POINTER(_SZ), ctypes.POINTER(_SZ)]),
    "rd_create": (_I, [_CFG, _PP]),
    "rd_attach": (_I, [_P, _P, _P]),
    "rd_destroy": (_I, [_P]),
    "rd_set_stream": (_I, [_P, _P]),
    "rd_set_field": (_I, [_P, _I, _P, _SZ]),
    "rd_step": (_I, [_P, _I64]),
    "rd_get_field": (_I, [_P, _I, _P, _SZ]),
    "rd_mass": (_I, [_P, _I, _DP]),
    "rd_sync": (_I, [_P]),
    "rd_wait": (_I, [_P, _I64]),
    "rd_step_count": (_I64, [_P]),
    "rd_set_step_count": (_I, [_P, _I64]),
    "rd_get_tuning": (_I, [_P, _TUN]),
    "rd_set_tuning": (_I, [_P, _TUN]),
    "rd_autotune": (_I, [_P, _TUN]),
    "rd_set_kernel": (_I, [_P, _I32]),
    "rd_get_kernel": (_I32, [_P]),
    "rd_launch_count": (_I64, [_P]),
    "rd_status_str": (ctypes.c_char_p, [_I]),
    "rd_last_error": (ctypes.c_char_p, [_P]),
    "rd_batch_create": (_I, [_I32, _I32, _PP]),
    "rd_batch_add": (_I, [_P, _P]),
    "rd_batch_remove": (_I, [_P, _P]),
    "rd_batch_size": (_I32, [_P]),
    "rd_batch_set_stream": (_I, [_P, _P]),
    "rd_batch_set_tuning": (_I, [_P, _TUN]),
    "rd_batch_step": (_I, [_P, _I64]),
    "rd_batch_step_each": (_I, [_P, ctypes.POINTER(ctypes.c_int64)]),
    "rd_batch_sync": (_I, [_P]),
    "rd_batch_destroy": (_I, [_P]),
    "rd_batch_launch_count": (_I64, [_P]),
    "rd_moments_noalloc": (_I, [_P, _I32, _I32, _I32, _I32, _I64, _P, _P]),
    "rd_debug_fail_alloc": (_I, [_I64]),
    "rd_debug_resident_stall": (_I, [_P, _I32]),
    "rd_set_resident_plan": (_I, [_P, _I32, _I32, _I32]),
    "rd_get_resident_plan": (_I, [_P, ctypes.POINTER(ctypes.c_int32)]),
    "rd_plane_bytes": (_SZ, [_P]),
    "rd_copy_planes": (_I, [_P, _I, _I, _I, _P, _SZ, _I32]),
    "rd_debug_bounds": (_I, [ctypes.POINTER(ctypes.c_uint64), _I32]),
}

_lib = None


def lib_path() -> str:
    """The library to load: the bounds-checked debug variant when the
    environment variable RD_BOUNDS_CHECK is 1, else the normal one."""
    if os.environ.get("RD_BOUNDS_CHECK") == "1":
        return _build.LIB_DEBUG
    return _build.LIB


def load():
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(
                f"CUDA library {path} is missing: build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class RdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(msg)
        self.status = status


def check(st, ctx=None, what=""):
    if st != RD_OK:
        lib = load()
        detail = lib.rd_last_error(ctx).decode()
        raise RdError(st, f"{what}: {lib.rd_status_str(st).decode()} ({detail})")
