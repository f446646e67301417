"""Python binding over the C ABI: ``Sim`` (one problem) and ``Batch``.

Argument marshalling only: every step, conversion and reduction runs in the
CUDA library.  PyTorch is used, when available, for device memory (contexts
created with ``torch_memory=True`` live in torch-allocated buffers attached
through ``rd_attach``) and for streams.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib as L

_PARAM_ORDER = {
    "diffusion": (),
    "brusselator": ("a", "b"),
    "ch_front": ("k", "M", "kappa"),
    "air": ("j", "k"),
    "turing": ("alpha", "beta", "gamma"),
    "ch_table1": ("k1", "k2", "lam", "eps", "gamma", "sigma"),
}


def make_config(cfg, storage="f32", force=False, no_alloc=False) -> L.RdConfig:
    """rd_config for a problem dictionary (``workloads`` format)."""
    lib = L.load()
    c = L.RdConfig()
    lib.rd_config_init(ctypes.byref(c))
    c.nx, c.ny, c.nz = cfg["shape"]
    c.nspecies = cfg["nspecies"]
    c.model = L.MODEL[cfg["model"]]
    c.storage = L.STORAGE[storage]
    c.h = cfg["h"]
    c.dt = cfg["dt"]
    for s in range(c.nspecies):
        for a in range(3):
            c.D[s][a] = cfg["D"][s][a]
        for f in range(6):
            c.bc[s][f] = L.BC[cfg["bc"][s][f]]
            c.bc_value[s][f] = cfg["bc_value"][s][f]
    for i, name in enumerate(_PARAM_ORDER[cfg["model"]]):
        c.params[i] = cfg["params"][name]
    w = cfg.get("wind")
    # the problem dictionaries name the plume's wind of Table 1 "table1"
    c.wind_kind = L.WIND[(("3d" if w["kind"] == "table1" else w["kind"]) if w else None)]
    if w and w["kind"] == "table1":
        # u = (ux, uy, uz_amp sin(t / uz_tau)), Table 1 row 4
        c.wind_vel[0], c.wind_vel[1], c.wind_vel[2] = w["ux"], w["uy"], w["uz_amp"]
        c.wind_tau = w["uz_tau"]
    else:
        c.wind_u0 = w["u0"] if w else 0.0
    src = cfg.get("source")
    if src:
        c.src_x, c.src_y, c.src_z = src["x"], src["y"], src["z"]
        c.src_species = src["species"]
        c.src_rate = src["rate"]
    else:
        c.src_species = -1
    c.stencil = cfg.get("stencil", 7)
    c.flags = (L.FLAG_FORCE if force else 0) | (L.FLAG_NO_ALLOC if no_alloc else 0)
    return c


def query_sizes(cfg, storage="f32"):
    lib = L.load()
    c = make_config(cfg, storage)
    a, b = ctypes.c_size_t(), ctypes.c_size_t()
    L.check(lib.rd_query_sizes(ctypes.byref(c), ctypes.byref(a), ctypes.byref(b)),
            None, "rd_query_sizes")
    return a.value, b.value


def _ptr(buf):
    """(address, keep-alive) of a float32 buffer: numpy array or torch tensor."""
    if isinstance(buf, np.ndarray):
        arr = np.ascontiguousarray(buf, dtype=np.float32)
        return arr.ctypes.data, arr
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(buf, torch.Tensor):
        if buf.dtype != torch.float32 or not buf.is_contiguous():
            raise ValueError("tensor must be contiguous float32")
        return buf.data_ptr(), buf
    raise TypeError(f"unsupported buffer type {type(buf)}")


class Sim:
    """One reaction-diffusion problem on the GPU.

    ``cfg``     problem dictionary (see ``workloads``)
    ``storage`` "f32" or "bf16"
    ``stream``  a torch.cuda.Stream, a raw cudaStream_t int, or None (the
                context's own stream)
    ``torch_memory``  allocate state and scratch with torch and attach them
    """

    def __init__(self, cfg, storage="f32", stream=None, torch_memory=False, force=False,
                 tuning=None):
        self.lib = L.load()
        self.cfg = cfg
        self.storage = storage
        self.shape = tuple(cfg["shape"])
        self.nspecies = cfg["nspecies"]
        self._keep = []
        conf = make_config(cfg, storage, force=force, no_alloc=torch_memory)
        ctx = ctypes.c_void_p()
        L.check(self.lib.rd_create(ctypes.byref(conf), ctypes.byref(ctx)), None, "rd_create")
        self.ctx = ctx
        try:
            if stream is not None:
                self.set_stream(stream)
            if torch_memory:
                import torch
                sb, xb = query_sizes(cfg, storage)
                st = torch.empty(sb + 256, dtype=torch.uint8, device="cuda")
                sc = torch.empty(xb + 256, dtype=torch.uint8, device="cuda")
                self._keep += [st, sc]
                a0 = (st.data_ptr() + 255) // 256 * 256
                a1 = (sc.data_ptr() + 255) // 256 * 256
                self._check(self.lib.rd_attach(self.ctx, ctypes.c_void_p(a0),
                                               ctypes.c_void_p(a1)), "rd_attach")
            if tuning is not None:
                self.set_tuning(**tuning)
        except BaseException:
            self.close()     # do not leak the context when setup fails
            raise

    # -- helpers
    def _check(self, st, what):
        L.check(st, self.ctx, what)

    @property
    def ncell(self):
        nx, ny, nz = self.shape
        return nx * ny * nz

    def set_stream(self, stream):
        handle = getattr(stream, "cuda_stream", stream)
        self._check(self.lib.rd_set_stream(self.ctx, ctypes.c_void_p(handle)), "rd_set_stream")

    # -- fields
    def set_field(self, s, values):
        addr, keep = _ptr(values)
        n = self.ncell
        count = keep.size if isinstance(keep, np.ndarray) else keep.numel()
        if count != n:
            raise ValueError(f"field has {count} values, the grid {n}")
        self._check(self.lib.rd_set_field(self.ctx, s, ctypes.c_void_p(addr), n), "rd_set_field")

    def set_fields(self, fields):
        for s in range(self.nspecies):
            self.set_field(s, fields[s])

    def get_field(self, s, out=None):
        nx, ny, nz = self.shape
        if out is None:
            out = np.empty((nz, ny, nx), dtype=np.float32)
        addr, keep = _ptr(out)
        self._check(self.lib.rd_get_field(self.ctx, s, ctypes.c_void_p(addr), self.ncell),
                    "rd_get_field")
        return out

    def get_fields(self):
        return np.stack([self.get_field(s) for s in range(self.nspecies)])

    # -- planes (z-slab exchange)
    @property
    def plane_bytes(self):
        """Bytes of one plane of one species in the context's layout."""
        return self.lib.rd_plane_bytes(self.ctx)

    def copy_planes(self, s, z0, k, buf, to_buf):
        """Copy planes z0 .. z0+k-1 of species s between the context and the
        device tensor ``buf`` (k * plane_bytes bytes, contiguous);
        asynchronous on the context's stream."""
        if not buf.is_cuda or not buf.is_contiguous():
            raise ValueError("buf must be a contiguous device tensor")
        nbytes = buf.numel() * buf.element_size()
        self._check(self.lib.rd_copy_planes(self.ctx, s, z0, k, ctypes.c_void_p(buf.data_ptr()),
                                            nbytes, 1 if to_buf else 0), "rd_copy_planes")

    # -- stepping
    def step(self, n):
        self._check(self.lib.rd_step(self.ctx, int(n)), "rd_step")

    def sync(self):
        self._check(self.lib.rd_sync(self.ctx), "rd_sync")

    def wait(self, timeout_ms):
        return self.lib.rd_wait(self.ctx, int(timeout_ms))

    def mass(self, s):
        out = (ctypes.c_double * 3)()
        st = self.lib.rd_mass(self.ctx, s, out)
        if st not in (L.RD_OK, L.RD_ENONFINITE):
            self._check(st, "rd_mass")
        return out[0], out[1], int(out[2])

    @property
    def steps_done(self):
        return self.lib.rd_step_count(self.ctx)

    @property
    def launches(self):
        return self.lib.rd_launch_count(self.ctx)

    # -- tuning
    def tuning(self):
        t = L.RdTuning()
        self._check(self.lib.rd_get_tuning(self.ctx, ctypes.byref(t)), "rd_get_tuning")
        return t.as_dict()

    def set_tuning(self, **kw):
        cur = self.tuning()
        cur.update(kw)
        t = L.RdTuning(cur["tsteps"], cur["tile_q"], cur["tile_y"], cur["zchunk"],
                       cur["graph"], cur.get("regcap", 0))
        self._check(self.lib.rd_set_tuning(self.ctx, ctypes.byref(t)), "rd_set_tuning")

    def set_kernel(self, name):
        """Step kernel: "march" (default), the paper's "shared" / "tiles"
        designs (ablation baselines; 19-point stencil, FP32, plain problems),
        or "resident" (many steps per cooperative launch for small grids held
        in L2; 7-point, no Cahn-Hilliard, no 3-D wind; same bits as march)."""
        self._check(self.lib.rd_set_kernel(self.ctx, L.KERNEL[name]), "rd_set_kernel")

    def set_resident_plan(self, K=0, tile_y=0, tile_z=0):
        """Resident kernel: K steps per round and tile_y x tile_z tiles
        (0 = the library's choice)."""
        self._check(self.lib.rd_set_resident_plan(self.ctx, K, tile_y, tile_z),
                    "rd_set_resident_plan")

    def resident_plan(self):
        out = (ctypes.c_int32 * 8)()
        self._check(self.lib.rd_get_resident_plan(self.ctx, out), "rd_get_resident_plan")
        return dict(zip(("K", "tile_y", "tile_z", "tiles", "ctas", "threads", "smem", "tma"),
                        list(out)))

    @property
    def kernel(self):
        code = self.lib.rd_get_kernel(self.ctx)
        return {v: k for k, v in L.KERNEL.items()}[code]

    def autotune(self):
        t = L.RdTuning()
        self._check(self.lib.rd_autotune(self.ctx, ctypes.byref(t)), "rd_autotune")
        return t.as_dict()

    # -- lifetime
    def close(self):
        if getattr(self, "ctx", None):
            self.lib.rd_destroy(self.ctx)
            self.ctx = None
            self._keep = []

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def member_counts(members, counts):
    """Step counts in member order for rd_batch_step_each; members missing
    from ``counts`` take 0 steps, and a key that is not a member is an
    error (its steps would otherwise be dropped without notice)."""
    ids = {id(m) for m in members}
    stray = [k for k in counts if id(k) not in ids]
    if stray:
        raise ValueError(f"{len(stray)} of the step counts name no member of the batch")
    return [int(counts.get(m, 0)) for m in members]


class Batch:
    """Contexts of one model and storage stepped by shared persistent launches."""

    def __init__(self, model, storage="f32", stream=None):
        self.lib = L.load()
        b = ctypes.c_void_p()
        L.check(self.lib.rd_batch_create(L.MODEL[model], L.STORAGE[storage], ctypes.byref(b)),
                None, "rd_batch_create")
        self.b = b
        self.members = []
        if stream is not None:
            self.set_stream(stream)

    def set_stream(self, stream):
        """Later steps run on ``stream`` (waits for the current one first)."""
        handle = getattr(stream, "cuda_stream", stream)
        L.check(self.lib.rd_batch_set_stream(self.b, ctypes.c_void_p(handle)), None,
                "rd_batch_set_stream")

    def add(self, sim: Sim):
        L.check(self.lib.rd_batch_add(self.b, sim.ctx), sim.ctx, "rd_batch_add")
        self.members.append(sim)

    def remove(self, sim: Sim):
        L.check(self.lib.rd_batch_remove(self.b, sim.ctx), sim.ctx, "rd_batch_remove")
        self.members.remove(sim)

    def set_tuning(self, tsteps=1, tile_q=16, tile_y=8, zchunk=32, graph=1, regcap=0):
        t = L.RdTuning(tsteps, tile_q, tile_y, zchunk, graph, regcap)
        L.check(self.lib.rd_batch_set_tuning(self.b, ctypes.byref(t)), None,
                "rd_batch_set_tuning")

    def step(self, n):
        L.check(self.lib.rd_batch_step(self.b, int(n)), None, "rd_batch_step")

    def step_each(self, counts):
        """Advance each member by its own count: ``counts`` maps a member
        Sim to its steps (members left out: 0; a Sim that is not a member:
        ValueError)."""
        arr = (ctypes.c_int64 * max(len(self.members), 1))(*member_counts(self.members, counts))
        L.check(self.lib.rd_batch_step_each(self.b, arr), None, "rd_batch_step_each")

    def sync(self):
        L.check(self.lib.rd_batch_sync(self.b), None, "rd_batch_sync")

    @property
    def launches(self):
        return self.lib.rd_batch_launch_count(self.b)

    def __len__(self):
        return self.lib.rd_batch_size(self.b)

    def close(self):
        if getattr(self, "b", None):
            self.lib.rd_batch_destroy(self.b)
            self.b = None
            self.members = []

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass
