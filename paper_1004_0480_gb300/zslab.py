"""Z-slab decomposition of one problem over ranks: the layout for a single
instance larger than one GPU's memory.

Each rank owns a contiguous range of z planes.  A side of the slab that
borders another rank (or wraps round, for periodic z) carries ``halo``
ghost planes: 1 for one step of the 7- or 19-point update, 2 for the
Cahn-Hilliard model, whose chained Laplacian reaches two planes.  A side on
a global non-periodic face has no ghost planes and keeps the global face
rule (zero flux, or a held layer).  After every step the ranks send their
outermost owned planes to their z neighbours, which refills the ghost
planes; the local step also updates the ghost planes (under a placeholder
zero-flux rule), and the exchange overwrites those values before any owned
cell reads them.  Every owned cell therefore sees exactly the neighbours it
has in the undivided grid, and the owned planes of all ranks equal the
undivided result bit for bit.

The step itself is a callable ``step_fn(fields, nsteps) -> fields`` on the
rank's local problem (``local_config``), so the decomposition does not
depend on the stepper.  Point-to-point messages go through
``torch.distributed`` (NCCL between GPUs, gloo on CPU); the fields are
float arrays of shape (S, nz_local, ny, nx).

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
    return 2 if cfg["model"] == "ch_front" else 1


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


def exchange(fields_local, p: SlabPlan, dist, torch):
    """Refill the ghost planes from the neighbours' outermost owned planes.

    Messages: the lowest ``lo_peer``-facing owned planes go to ``lo_peer``
    (tag 1: they become its upper ghost planes), the highest go to
    ``hi_peer`` (tag 0: its lower ghost planes).  Receives are posted
    before sends; with two ranks and periodic z both messages go to the
    same peer and are told apart by their tags."""
    if p.world == 1:
        return fields_local
    f = torch.from_numpy(fields_local) if isinstance(fields_local, np.ndarray) else fields_local
    own = p.owned
    reqs, recv = [], []
    if p.lo:
        buf = torch.empty_like(f[:, :p.lo]).contiguous()
        reqs.append(dist.irecv(buf, src=p.lo_peer, tag=0))
        recv.append((slice(0, p.lo), buf))
    if p.hi:
        buf = torch.empty_like(f[:, f.shape[1] - p.hi:]).contiguous()
        reqs.append(dist.irecv(buf, src=p.hi_peer, tag=1))
        recv.append((slice(f.shape[1] - p.hi, f.shape[1]), buf))
    sends = []
    if p.lo:
        sends.append(f[:, own.start:own.start + p.lo].contiguous())
        reqs.append(dist.isend(sends[-1], dst=p.lo_peer, tag=1))
    if p.hi:
        sends.append(f[:, own.stop - p.hi:own.stop].contiguous())
        reqs.append(dist.isend(sends[-1], dst=p.hi_peer, tag=0))
    for r in reqs:
        r.wait()
    for sl, buf in recv:
        f[:, sl] = buf
    return fields_local


def run(fields_local, p: SlabPlan, nsteps: int, step_fn, dist, torch):
    """Advance the rank's slab by ``nsteps`` steps, one exchange per step.
    ``fields_local`` must hold valid ghost planes (``scatter``, or a
    preceding ``run``)."""
    f = fields_local
    for _ in range(int(nsteps)):
        f = np.ascontiguousarray(step_fn(f, 1))
        f = exchange(f, p, dist, torch)
    return f
