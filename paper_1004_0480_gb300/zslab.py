"""Z-slab decomposition of one problem over ranks: the layout for a single
instance larger than one GPU's memory.

Each rank owns a contiguous range of z planes.  A side of the slab that
borders another rank (or wraps round, for periodic z) carries ``halo``
ghost planes: 1 for one step of the 7- or 19-point update, 2 for the
Cahn-Hilliard models, whose chained Laplacian reaches two planes.  A side on
a global non-periodic face has no ghost planes and keeps the global face
rule (zero flux, or a held layer).  After every step the ranks send their
outermost owned planes to their z neighbours, which refills the ghost
planes; the local step also updates the ghost planes (under a placeholder
zero-flux rule), and the exchange overwrites those values before any owned
cell reads them.  Every owned cell therefore sees exactly the neighbours it
has in the undivided grid, and the owned planes of all ranks equal the
undivided result bit for bit.

A rank's slab is an object with ``read(z0, k)``, ``empty(k)``,
``write(z0, k, buf)`` and ``step(n)``: ``HostSlab`` holds float arrays and
steps them with any callable (the CPU tests use the FP64 oracle);
``DeviceSlab`` keeps the fields on the rank's GPU in a context of the CUDA
library, moves ghost planes with ``rd_copy_planes`` (device to device, the
context's own layout) and steps with ``rd_step``.  ``exchange`` moves the
planes with ``torch.distributed`` point-to-point messages, posted as one
batch in the same order on every rank (NCCL between GPUs, into each
receiving GPU's own buffers; gloo on CPU);
``exchange_local`` moves them between slabs held by one process (the same
messages, no collective).  ``owned_moments`` reduces the owned planes in
FP64 and sums the ranks' results with an FP64 all-reduce.

Not supported: the logarithmic wind profile (its u(z) depends on the global
plane index and nz, which a local problem does not know) and slabs thinner
than the halo.
"""
from __future__ import annotations

import copy
from dataclasses import dataclass

import numpy as np

_Z_LO, _Z_HI = 4, 5          # face indices of -z and +z


def split(nz: int, world: int) -> list[tuple[int, int]]:
    """Balanced contiguous z ranges [z0, z1) of ``world`` ranks."""
    if world < 1 or nz < world:
        raise ValueError(f"cannot split {nz} planes over {world} ranks")
    base, extra = divmod(nz, world)
    out, z = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((z, z + n))
        z += n
    return out


@dataclass
class SlabPlan:
    rank: int
    world: int
    z0: int                  # first owned global plane
    z1: int                  # one past the last owned plane
    lo: int                  # ghost planes below the owned range (0 at a global face)
    hi: int                  # ghost planes above
    lo_peer: int | None      # rank that owns the planes below (None: global face)
    hi_peer: int | None
    cfg: dict                # the rank's local problem

    @property
    def owned(self) -> slice:
        """Owned planes within the local z axis."""
        return slice(self.lo, self.lo + (self.z1 - self.z0))


def halo_width(cfg) -> int:
    return 2 if cfg["model"] in ("ch_front", "ch_table1") else 1


def plan(cfg, world: int, rank: int) -> SlabPlan:
    """The slab of ``rank`` and its local problem."""
    nx, ny, nz = cfg["shape"]
    S = cfg["nspecies"]
    w = halo_width(cfg)
    ranges = split(nz, world)
    z0, z1 = ranges[rank]
    if min(b - a for a, b in ranges) < w and world > 1:
        raise ValueError(f"every slab needs at least {w} planes")
    wind = cfg.get("wind")
    if wind and wind["kind"] == "log":
        raise ValueError("the logarithmic wind profile needs the global plane index")
    periodic_z = cfg["bc"][0][_Z_LO] == "periodic"
    if world == 1:
        lo_peer = hi_peer = None
    else:
        lo_peer = rank - 1 if rank > 0 else (world - 1 if periodic_z else None)
        hi_peer = rank + 1 if rank < world - 1 else (0 if periodic_z else None)
    lo = w if lo_peer is not None else 0
    hi = w if hi_peer is not None else 0

    local = copy.deepcopy(cfg)
    local["shape"] = (nx, ny, (z1 - z0) + lo + hi)
    local["name"] = f"{cfg.get('name', 'problem')}_slab{rank}of{world}"
    bc = [list(b) for b in cfg["bc"]]
    for s in range(S):
        if periodic_z and world > 1:
            bc[s][_Z_LO] = bc[s][_Z_HI] = "neumann"
        if lo:
            bc[s][_Z_LO] = "neumann"     # placeholder: ghost planes are overwritten
        if hi:
            bc[s][_Z_HI] = "neumann"
    local["bc"] = bc
    src = cfg.get("source")
    if src:
        if z0 <= src["z"] < z1:
            local["source"] = dict(src, z=src["z"] - z0 + lo)
        else:
            local["source"] = None
    return SlabPlan(rank, world, z0, z1, lo, hi, lo_peer, hi_peer, local)


def scatter(fields_global, p: SlabPlan):
    """The rank's local fields, ghost planes included, cut from the undivided
    fields (S, nz, ny, nx)."""
    nz = fields_global.shape[1]
    idx = np.arange(p.z0 - p.lo, p.z1 + p.hi) % nz
    return np.ascontiguousarray(fields_global[:, idx])


def owned(fields_local, p: SlabPlan):
    return fields_local[:, p.owned]


def messages(p: SlabPlan):
    """The plane transfers of one exchange, as (peer, tag, local z0, k):
    the lowest owned planes go to ``lo_peer`` with tag 1 (they become its
    upper ghost planes), the highest to ``hi_peer`` with tag 0 (its lower
    ghost planes); receives mirror them.  With two ranks and periodic z both
    messages go to the same peer and are told apart by their tags."""
    if p.world == 1:
        return [], []
    nzl = p.cfg["shape"][2]
    own = p.owned
    sends, recvs = [], []
    if p.lo:
        recvs.append((p.lo_peer, 0, 0, p.lo))
        sends.append((p.lo_peer, 1, own.start, p.lo))
    if p.hi:
        recvs.append((p.hi_peer, 1, nzl - p.hi, p.hi))
        sends.append((p.hi_peer, 0, own.stop - p.hi, p.hi))
    return sends, recvs


def posting_order(p: SlabPlan):
    """The exchange's sends and receives in the order every rank posts them:
    by peer, then tag.  A backend that pairs the messages between two ranks
    by their order and ignores tags (NCCL) then matches each send with the
    receive meant for it, also where both neighbours are one rank (two
    ranks, periodic z: a rank's lowest and highest owned planes both go to
    the other rank)."""
    sends, recvs = messages(p)
    return sorted(sends), sorted(recvs)


def exchange(slab, p: SlabPlan, dist):
    """Refill the slab's ghost planes from the neighbours' outermost owned
    planes by point-to-point messages, posted as one batch
    (``batch_isend_irecv``: a single NCCL group, so no rank's receive waits
    behind its own sends; with NCCL the current CUDA device must be the
    rank's own)."""
    sends, recvs = posting_order(p)
    if not sends and not recvs:
        return
    ops, landed = [], []
    for peer, tag, z0, k in recvs:
        buf = slab.empty(k)
        ops.append(dist.P2POp(dist.irecv, buf, peer, tag=tag))
        landed.append((z0, k, buf))
    for peer, tag, z0, k in sends:
        ops.append(dist.P2POp(dist.isend, slab.read(z0, k), peer, tag=tag))
    for r in dist.batch_isend_irecv(ops):
        r.wait()
    for z0, k, buf in landed:
        slab.write(z0, k, buf)


def exchange_local(slabs, plans):
    """The same exchange between the slabs of all ranks held by one process
    (every outgoing plane is read before any ghost plane is written)."""
    mail = {}
    for r, (slab, p) in enumerate(zip(slabs, plans)):
        for peer, tag, z0, k in messages(p)[0]:
            mail[(r, peer, tag)] = slab.read(z0, k)
    for r, (slab, p) in enumerate(zip(slabs, plans)):
        for peer, tag, z0, k in messages(p)[1]:
            slab.write(z0, k, mail[(peer, r, tag)])


def run_slab(slab, p: SlabPlan, nsteps: int, dist):
    """Advance the rank's slab by ``nsteps`` steps, one exchange per step.
    The slab must hold valid ghost planes (its initial fields cut by
    ``scatter``, or a preceding run)."""
    for _ in range(int(nsteps)):
        slab.step(1)
        exchange(slab, p, dist)


def run_local(slabs, plans, nsteps: int):
    """``run_slab`` for the slabs of all ranks held by one process."""
    for _ in range(int(nsteps)):
        for slab in slabs:
            slab.step(1)
        exchange_local(slabs, plans)


class HostSlab:
    """A slab as a float array (S, nz_local, ny, nx) stepped by
    ``step_fn(fields, nsteps) -> fields`` (on the CPU); ``plan`` names the
    owned planes for ``moments``."""

    def __init__(self, fields_local, step_fn, plan: SlabPlan | None = None):
        import torch
        self._torch = torch
        self.fields = np.ascontiguousarray(fields_local)
        self.step_fn = step_fn
        self.plan = plan

    def moments(self, s):
        """FP64 (sum, sum of squares, non-finite count) of species ``s`` over
        the owned planes."""
        f = np.asarray(self.fields[s, self.plan.owned], dtype=np.float64)
        ok = np.isfinite(f)
        return self._torch.tensor([f[ok].sum(), (f[ok] ** 2).sum(), float((~ok).sum())],
                                  dtype=self._torch.float64)

    def read(self, z0, k):
        return self._torch.from_numpy(np.ascontiguousarray(self.fields[:, z0:z0 + k]))

    def empty(self, k):
        S, _, ny, nx = self.fields.shape
        return self._torch.empty((S, k, ny, nx), dtype=self._torch.from_numpy(self.fields[:0]).dtype)

    def write(self, z0, k, buf):
        self.fields[:, z0:z0 + k] = buf.numpy()

    def step(self, n):
        self.fields = np.ascontiguousarray(self.step_fn(self.fields, n))


class DeviceSlab:
    """A slab kept on the rank's GPU: a context of the CUDA library for the
    local problem, on torch's current stream (so NCCL messages and the
    plane copies are ordered with the steps).  Ghost planes move as raw
    planes of the context's layout (storage type, row pitch), one
    device-to-device copy per species and side."""

    def __init__(self, p: SlabPlan, storage="f32", tuning=None):
        import torch

        from .sim import Sim
        self._torch = torch
        self.plan = p
        self.storage = storage
        self.sim = Sim(p.cfg, storage, stream=torch.cuda.current_stream(), tuning=tuning)
        self.S = p.cfg["nspecies"]
        self.pb = self.sim.plane_bytes

    def set_fields(self, fields_local):
        self.sim.set_fields(fields_local)

    def empty(self, k):
        return self._torch.empty(self.S * k * self.pb, dtype=self._torch.uint8, device="cuda")

    def read(self, z0, k):
        buf = self.empty(k)
        n = k * self.pb
        for s in range(self.S):
            self.sim.copy_planes(s, z0, k, buf[s * n:(s + 1) * n], to_buf=True)
        return buf

    def write(self, z0, k, buf):
        n = k * self.pb
        for s in range(self.S):
            self.sim.copy_planes(s, z0, k, buf[s * n:(s + 1) * n], to_buf=False)

    def step(self, n):
        self.sim.step(n)

    def owned_fields(self):
        return self.sim.get_fields()[:, self.plan.owned]

    def moments(self, s):
        """FP64 (sum, sum of squares, non-finite count) of species ``s`` over
        the owned planes (the library's allocation-free reduction on a copy
        of those planes)."""
        import ctypes

        from . import _lib as L
        p = self.plan
        k = p.z1 - p.z0
        nx, ny, _ = p.cfg["shape"]
        buf = self._torch.empty(k * self.pb, dtype=self._torch.uint8, device="cuda")
        self.sim.copy_planes(s, p.owned.start, k, buf, to_buf=True)
        out = self._torch.zeros(3, dtype=self._torch.float64, device="cuda")
        eb = 2 if self.storage == "bf16" else 4
        st = self.sim.lib.rd_moments_noalloc(
            ctypes.c_void_p(buf.data_ptr()), L.STORAGE[self.storage], nx, ny, k,
            self.pb // (ny * eb), ctypes.c_void_p(out.data_ptr()),
            ctypes.c_void_p(self._torch.cuda.current_stream().cuda_stream))
        L.check(st, None, "rd_moments_noalloc")
        return out

    def close(self):
        self.sim.close()


def owned_moments(slab, s, dist=None):
    """The whole grid's FP64 moments of species ``s``: each rank's owned
    planes, summed over ranks by an FP64 all-reduce."""
    out = slab.moments(s)
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(out)
    return out


def run(fields_local, p: SlabPlan, nsteps: int, step_fn, dist, torch=None):
    """Advance a host slab (float arrays, ghost planes included, stepped by
    ``step_fn``) by ``nsteps`` steps; returns the new local fields."""
    slab = HostSlab(fields_local, step_fn)
    run_slab(slab, p, nsteps, dist)
    return slab.fields
