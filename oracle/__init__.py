"""FP64 CPU oracle for the reaction-diffusion step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the benchmark's CPU-baseline / reference leg may import this package.  It
shares no code with the CUDA path (``paper_1004_0480_gb300``) and does not
import it.

Two independent implementations of the same definition:

* ``run``     -- the C stepper (``rd_oracle.c``), FP64, single-threaded;
* ``np_run``  -- a NumPy restatement (``np_oracle.py``) used to cross-check it.

Both take a problem dictionary (the shape produced by
``paper_1004_0480_gb300.workloads``, plain data only) and initial fields of
shape (S, nz, ny, nx).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from .np_oracle import np_run  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liborc.so")
_SRC = os.path.join(_HERE, "rd_oracle.c")
_HDR = os.path.join(_HERE, "rd_oracle.h")

MAXS = 4
_BC = {"neumann": 0, "periodic": 1, "dirichlet": 2}
_MODEL = {"diffusion": 0, "brusselator": 1, "ch_front": 2, "air": 3, "turing": 4, "ch_table1": 5}
_WIND = {None: 0, "log": 1, "const": 2, "table1": 3}


class OrcProblem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("ns", ctypes.c_int32), ("model", ctypes.c_int32),
        ("wind_kind", ctypes.c_int32),
        ("h", ctypes.c_double), ("dt", ctypes.c_double),
        ("D", (ctypes.c_double * 3) * MAXS),
        ("bc", (ctypes.c_int32 * 6) * MAXS),
        ("bc_value", (ctypes.c_double * 6) * MAXS),
        ("p", ctypes.c_double * 8),
        ("wind_u0", ctypes.c_double),
        ("src_x", ctypes.c_int32), ("src_y", ctypes.c_int32),
        ("src_z", ctypes.c_int32), ("src_species", ctypes.c_int32),
        ("src_rate", ctypes.c_double),
        ("stencil", ctypes.c_int32), ("pad0", ctypes.c_int32),
        ("w3", ctypes.c_double * 4),
        ("n0", ctypes.c_int64),
    ]


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc into ``oracle/_build/liborc.so``."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC),
                                                   os.path.getmtime(_HDR))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-ffp-contract=off", "-fPIC",
           "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        lib.orc_run.argtypes = [ctypes.POINTER(OrcProblem),
                                ctypes.POINTER(ctypes.c_double), ctypes.c_int64]
        lib.orc_run.restype = ctypes.c_int
        lib.orc_wind.argtypes = [ctypes.POINTER(OrcProblem), ctypes.c_int]
        lib.orc_wind.restype = ctypes.c_double
        _lib = lib
    return _lib


_PARAM_ORDER = {
    "diffusion": (),
    "brusselator": ("a", "b"),
    "ch_front": ("k", "M", "kappa"),
    "air": ("j", "k"),
    "turing": ("alpha", "beta", "gamma"),
    "ch_table1": ("k1", "k2", "lam", "eps", "gamma", "sigma"),
}


def make_problem(cfg) -> OrcProblem:
    p = OrcProblem()
    p.nx, p.ny, p.nz = cfg["shape"]
    p.ns = cfg["nspecies"]
    p.model = _MODEL[cfg["model"]]
    p.h = cfg["h"]
    p.dt = cfg["dt"]
    for s in range(p.ns):
        for a in range(3):
            p.D[s][a] = cfg["D"][s][a]
        for f in range(6):
            p.bc[s][f] = _BC[cfg["bc"][s][f]]
            p.bc_value[s][f] = cfg["bc_value"][s][f]
    for i, name in enumerate(_PARAM_ORDER[cfg["model"]]):
        p.p[i] = cfg["params"][name]
    w = cfg.get("wind")
    p.wind_kind = _WIND[w["kind"] if w else None]
    p.wind_u0 = w.get("u0", 0.0) if w else 0.0
    if w and w["kind"] == "table1":
        p.w3[0], p.w3[1], p.w3[2], p.w3[3] = w["ux"], w["uy"], w["uz_amp"], w["uz_tau"]
    src = cfg.get("source")
    if src:
        p.src_x, p.src_y, p.src_z = src["x"], src["y"], src["z"]
        p.src_species = src["species"]
        p.src_rate = src["rate"]
    else:
        p.src_species = -1
    p.stencil = cfg.get("stencil", 7)
    return p


def run(cfg, fields, nsteps, n0=0) -> np.ndarray:
    """Advance ``fields`` (S, nz, ny, nx) by ``nsteps`` steps in FP64 with
    the C oracle, the first step having index ``n0`` (its time is n0 dt);
    returns a new float64 array."""
    lib = _load()
    nx, ny, nz = cfg["shape"]
    st = np.ascontiguousarray(np.asarray(fields, dtype=np.float64)).copy()
    if st.shape != (cfg["nspecies"], nz, ny, nx):
        raise ValueError(f"fields shape {st.shape} does not match the problem")
    p = make_problem(cfg)
    p.n0 = int(n0)
    rc = lib.orc_run(ctypes.byref(p),
                     st.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                     int(nsteps))
    if rc != 0:
        raise ValueError("oracle rejected the problem")
    return st


def wind(cfg, z) -> float:
    return _load().orc_wind(ctypes.byref(make_problem(cfg)), int(z))
