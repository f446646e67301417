"""Seeded synthetic workloads: problem parameters and initial fields.

This module holds no arithmetic of the method (no Laplacian, reaction,
advection or time update).  It only states the problems (grid, species,
coefficients, boundary kinds, seeds) and draws their initial fields, so both
the CUDA path and the CPU oracle can be fed the same inputs.

Problems follow the four families of the paper's Table 1 (inert diffusion,
Turing pattern, Cahn-Hilliard phase separation behind a front, atmospheric
advection-diffusion), in the concrete parameterisation used for the
benchmarks here:

* ``diffusion_blob``   inert diffusion, 1 species, Neumann faces, uniform noise
  plus a centred Gaussian blob (amplitude 10, sigma 6).
* ``brusselator``      Brusselator Turing system, 2 species, periodic.
* ``ch_front``         a + b -> c behind a front held on the z = 0 face, with
  c following a Cahn-Hilliard equation (two chained Laplacians).
* ``air``              NO / NO2 / O3 photochemistry with a log wind profile in
  x, per-axis diffusivity and a point source of NO.

Random numbers come from a counter-based splitmix64 generator (Steele, Lea
and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014;
the 64-bit finaliser constants are the published ones), keyed by
(seed, species, linear cell index), so any cell's draw is reproducible on
any machine without generating the others.
"""
from __future__ import annotations

import copy

import numpy as np

# --------------------------------------------------------------------------
# counter-based uniform numbers
# --------------------------------------------------------------------------
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_SPECIES_KEY = np.uint64(0xC2B2AE3D27D4EB4F)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(counter: np.ndarray) -> np.ndarray:
    """splitmix64 output function applied to an array of uint64 counters."""
    with np.errstate(over="ignore"):
        z = counter.astype(np.uint64, copy=True)
        z += _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z ^= z >> np.uint64(31)
    return z


def uniform01(seed: int, species: int, n: int, start: int = 0) -> np.ndarray:
    """U[0,1) draws for cells ``start .. start+n-1`` of one species (float64).

    counter = seed*GOLDEN xor species*KEY, plus the linear cell index;
    U = (splitmix64(counter) >> 11) * 2**-53.
    """
    with np.errstate(over="ignore"):
        base = (np.uint64(seed) * _GOLDEN) ^ (np.uint64(species) * _SPECIES_KEY)
        ctr = base + np.arange(start, start + n, dtype=np.uint64)
    z = splitmix64(ctr)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


# --------------------------------------------------------------------------
# problem statements
# --------------------------------------------------------------------------
NEU, PER, DIR = "neumann", "periodic", "dirichlet"
# face order used everywhere: -x, +x, -y, +y, -z, +z
FACES = ("-x", "+x", "-y", "+y", "-z", "+z")


def _bc(kind, ns):
    return [[kind] * 6 for _ in range(ns)]


def diffusion_blob(n=64, steps=100, dt=0.1, D=1.0, h=1.0, seed=0, shape=None):
    """Inert diffusion of one species from a centred blob (Table 1, row 1)."""
    nx, ny, nz = shape if shape is not None else (n, n, n)
    return dict(name=f"diffusion_blob_{nx}x{ny}x{nz}", model="diffusion",
                shape=(nx, ny, nz), nspecies=1, h=h, dt=dt,
                D=[[D, D, D]], bc=_bc(NEU, 1), bc_value=[[0.0] * 6],
                params={}, source=None, wind=None, steps=steps, seed=seed,
                init="blob")


def brusselator(n=256, steps=10000, dt=0.005, a=3.0, b=9.0, Du=2.0, Dv=16.0,
                h=1.0, seed=1, bc=PER, shape=None):
    """Brusselator Turing system, 2 species (Table 1, row 2 family)."""
    nx, ny, nz = shape if shape is not None else (n, n, n)
    return dict(name=f"brusselator_{nx}x{ny}x{nz}", model="brusselator",
                shape=(nx, ny, nz), nspecies=2, h=h, dt=dt,
                D=[[Du] * 3, [Dv] * 3], bc=_bc(bc, 2), bc_value=[[0.0] * 6] * 2,
                params=dict(a=a, b=b), source=None, wind=None, steps=steps,
                seed=seed, init="brusselator")


def ch_front(n=64, steps=2000, dt=0.01, Da=1.0, Db=0.1, k=1.0, M=0.1,
             kappa=1.0, a_front=10.0, h=1.0, seed=2, shape=None):
    """Reaction front a + b -> c with Cahn-Hilliard phase separation of c
    (Table 1, row 3 family).  Species a is held at ``a_front`` on the z = 0
    face; all other faces are zero-flux."""
    nx, ny, nz = shape if shape is not None else (n, n, n)
    bc = _bc(NEU, 3)
    bcv = [[0.0] * 6 for _ in range(3)]
    bc[0][4] = DIR
    bcv[0][4] = a_front
    return dict(name=f"ch_front_{nx}x{ny}x{nz}", model="ch_front",
                shape=(nx, ny, nz), nspecies=3, h=h, dt=dt,
                D=[[Da] * 3, [Db] * 3, [0.0] * 3], bc=bc, bc_value=bcv,
                params=dict(k=k, M=M, kappa=kappa), source=None, wind=None,
                steps=steps, seed=seed, init="ch_front")


def ch_table1(n=192, steps=20000, dt=0.02, D1=1.0, D2=1.0, k1=0.2, k2=0.005, lam=1.0,
              eps=1.0, gamma=1.0, sigma=1.0, c1_front=10.0, h=1.0, seed=7, shape=None,
              stencil=19):
    """Phase separation behind a chemical front, Table 1, row 3, with its
    parameters: c1 + c2 -> c3 (k1), the sink k2 c1 c3 of c1 and c3, and
    dc3/dt += -lambda Lap(eps c3 - gamma c3^3 + sigma Lap c3); c3 has no
    Fickian term.  c1 is held at 10 on the x = 0 layer, every other face is
    zero flux; c1 = 0, c2 = 1, c3 = -1 at the start.  The paper's stencil
    is the 19-point one, and its dt = 0.02 is within the explicit bound only
    for that stencil."""
    nx, ny, nz = shape if shape is not None else (n, n, n)
    bc = _bc(NEU, 3)
    bcv = [[0.0] * 6 for _ in range(3)]
    bc[0][0] = DIR
    bcv[0][0] = c1_front
    return dict(name=f"ch_table1_{nx}x{ny}x{nz}", model="ch_table1", shape=(nx, ny, nz),
                nspecies=3, h=h, dt=dt, D=[[D1] * 3, [D2] * 3, [0.0] * 3], bc=bc, bc_value=bcv,
                params=dict(k1=k1, k2=k2, lam=lam, eps=eps, gamma=gamma, sigma=sigma),
                source=None, wind=None, steps=steps, seed=seed, init="ch_table1",
                stencil=stencil)


def turing(n=192, steps=20000, dt=5.0e-4, D1=5.0e-5, D2=5.0e-3, h=6.2e-3, alpha=0.5,
           beta=0.09, gamma=26.0, sigma=5.0e-4, seed=5, shape=None, stencil=7):
    """Activator-inhibitor Turing system of Table 1, row 2, with its
    parameters: dc1/dt = D1 Lap c1 + c1 - c1^3 - c2,
    dc2/dt = D2 Lap c2 + gamma (c1 - alpha c2 - beta); zero flux; both
    species start at 1 + U(-sigma, sigma)."""
    nx, ny, nz = shape if shape is not None else (n, n, n)
    return dict(name=f"turing_{nx}x{ny}x{nz}", model="turing", shape=(nx, ny, nz),
                nspecies=2, h=h, dt=dt, D=[[D1] * 3, [D2] * 3], bc=_bc(NEU, 2),
                bc_value=[[0.0] * 6] * 2, params=dict(alpha=alpha, beta=beta, gamma=gamma),
                source=None, wind=None, steps=steps, seed=seed, init="turing",
                sigma=sigma, stencil=stencil)


def air(shape=(512, 512, 64), steps=5000, dt=0.2, Kh=0.1, Kz=0.02, j=0.5,
        k=2.0, src=(64, 256, 2), src_rate=1.0, h=1.0, seed=3, wind_u0=1.0):
    """NO/NO2/O3 advection-diffusion-reaction (Table 1, row 4 family)."""
    nx, ny, nz = shape
    return dict(name=f"air_{nx}x{ny}x{nz}", model="air", shape=(nx, ny, nz),
                nspecies=3, h=h, dt=dt, D=[[Kh, Kh, Kz]] * 3,
                bc=_bc(NEU, 3), bc_value=[[0.0] * 6] * 3,
                params=dict(j=j, k=k),
                source=dict(x=src[0], y=src[1], z=src[2], species=0,
                            rate=src_rate),
                wind=dict(kind="log", u0=wind_u0), steps=steps, seed=seed,
                init="air")


def plume(shape=(144, 144, 384), steps=20000, dt=5.0, D=100.0, h=100.0, ux=5.0, uy=1.0,
          uz_amp=5.0, uz_tau=500.0, E=10.0, src=None, seed=6):
    """Inert plume of Table 1, row 4, with its parameters: dc/dt =
    -div(u c) + D Lap c + E, u = (5, 1, 5 sin(t / 500 s)) m/s, D = 100 m^2/s,
    h = 100 m, dt = 5 s, a point emission E = 10 per second, c0 = 0, zero
    flux; the 144 x 144 x 384 grid of Figure 7.  The paper does not place
    the source: by default a quarter of the way along x, centred in y, an
    eighth of the way up z."""
    nx, ny, nz = shape
    sx, sy, sz = src if src is not None else (nx // 4, ny // 2, nz // 8)
    return dict(name=f"plume_{nx}x{ny}x{nz}", model="diffusion", shape=(nx, ny, nz),
                nspecies=1, h=h, dt=dt, D=[[D] * 3], bc=_bc(NEU, 1), bc_value=[[0.0] * 6],
                params={}, source=dict(x=sx, y=sy, z=sz, species=0, rate=E),
                wind=dict(kind="table1", ux=ux, uy=uy, uz_amp=uz_amp, uz_tau=uz_tau),
                steps=steps, seed=seed, init="zero")


def with_(cfg, **kw):
    """Copy of a problem with some entries replaced."""
    c = copy.deepcopy(cfg)
    c.update(kw)
    return c


# --------------------------------------------------------------------------
# initial fields
# --------------------------------------------------------------------------
def initial_fields(cfg, seed=None, dtype=np.float32):
    """Initial fields of a problem, shape (S, nz, ny, nx), x fastest.

    Drawn in float64 and rounded once to ``dtype``: the oracle and the CUDA
    path both start from these rounded values.
    """
    nx, ny, nz = cfg["shape"]
    ncell = nx * ny * nz
    s = cfg["seed"] if seed is None else seed
    S = cfg["nspecies"]
    out = np.empty((S, nz, ny, nx), dtype=np.float64)
    kind = cfg["init"]
    if kind == "blob":
        u = uniform01(s, 0, ncell).reshape(nz, ny, nx)
        z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx),
                              indexing="ij")
        cx, cy, cz = (nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0
        r2 = (x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2
        out[0] = u + 10.0 * np.exp(-r2 / (2.0 * 6.0 ** 2))
    elif kind == "brusselator":
        a, b = cfg["params"]["a"], cfg["params"]["b"]
        base = (a, b / a)
        for sp in range(2):
            u = uniform01(s, sp, ncell).reshape(nz, ny, nx)
            out[sp] = base[sp] * (1.0 + 0.01 * (2.0 * u - 1.0))
    elif kind == "ch_front":
        out[0] = 0.0
        out[0, 0, :, :] = cfg["bc_value"][0][4]
        out[1] = 1.0
        u = uniform01(s, 2, ncell).reshape(nz, ny, nx)
        out[2] = 0.005 * (2.0 * u - 1.0)
    elif kind == "air":
        base = (0.01, 0.01, 1.0)
        for sp in range(3):
            u = uniform01(s, sp, ncell).reshape(nz, ny, nx)
            out[sp] = base[sp] * (1.0 + 0.01 * (2.0 * u - 1.0))
    elif kind == "turing":
        sig = cfg["sigma"]
        for sp in range(2):
            u = uniform01(s, sp, ncell).reshape(nz, ny, nx)
            out[sp] = 1.0 + sig * (2.0 * u - 1.0)
    elif kind == "zero":
        out[:] = 0.0
    elif kind == "ch_table1":
        out[0] = 0.0
        out[0, :, :, 0] = cfg["bc_value"][0][0]
        out[1] = 1.0
        out[2] = -1.0
    elif kind == "uniform_noise":
        for sp in range(S):
            out[sp] = uniform01(s, sp, ncell).reshape(nz, ny, nx)
    else:
        raise ValueError(f"unknown initial condition {kind!r}")
    return out.astype(dtype)


# --------------------------------------------------------------------------
# the benchmark workloads at their full sizes
# --------------------------------------------------------------------------
def cfg_diffusion_64():
    """64^3 inert diffusion, dt 0.1, 100 steps, seed 0."""
    return diffusion_blob(64, steps=100, dt=0.1, seed=0)


def cfg_brusselator_256():
    """256^3 periodic Brusselator, a=3, b=9, Du=2, Dv=16, dt 0.005,
    10 000 steps, seed 1."""
    return brusselator(256, steps=10000, dt=0.005, seed=1)


def cfg_brusselator_256_19pt():
    """The 256^3 Brusselator with the paper's 19-point Laplacian (eqs. (3)-(4))."""
    return with_(cfg_brusselator_256(), stencil=19,
                 name="brusselator_256x256x256_19pt")


def batch_sizes_ch(count=32, lo=48, hi=192, seed=2):
    """Uneven cube edges for the batched front workload (seeded)."""
    rng = np.random.default_rng(seed)
    return [int(v) for v in rng.integers(lo, hi + 1, size=count)]


def cfg_ch_front_batch(count=32, steps=2000):
    """32 front instances, edges uniform in 48..192, dt 0.01, 2000 steps;
    instance i is seeded 2 + 1000 i."""
    return [ch_front(n, steps=steps, seed=2 + 1000 * i)
            for i, n in enumerate(batch_sizes_ch(count))]


def cfg_air_512():
    """512x512x64 NO/NO2/O3 air problem, dt 0.2, 5000 steps, seed 3."""
    return air((512, 512, 64), steps=5000, seed=3)


SERVE_EDGES = (32, 64, 96, 128, 192, 256, 384)
SERVE_KINDS = ("diffusion", "brusselator", "ch_front")


def serving_requests(count=500, rate_per_s=50.0, seed=4, edges=SERVE_EDGES,
                     steps_lo=100, steps_hi=5000):
    """Poisson arrival stream of mixed requests.

    Each request: arrival time (s), kinetics family (uniform over the three
    families), cube edge (uniform over ``edges``), step count (uniform
    integer in [steps_lo, steps_hi]) and its own field seed.
    """
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=count)
    t = np.cumsum(gaps) - gaps[0]
    kinds = rng.integers(0, len(SERVE_KINDS), size=count)
    ns = rng.integers(0, len(edges), size=count)
    steps = rng.integers(steps_lo, steps_hi + 1, size=count)
    reqs = []
    for i in range(count):
        kind = SERVE_KINDS[int(kinds[i])]
        n = int(edges[int(ns[i])])
        st = int(steps[i])
        fseed = 100000 + i
        if kind == "diffusion":
            cfg = diffusion_blob(n, steps=st, dt=0.1, seed=fseed)
        elif kind == "brusselator":
            cfg = brusselator(n, steps=st, dt=0.005, seed=fseed)
        else:
            cfg = ch_front(n, steps=st, seed=fseed)
        reqs.append(dict(id=i, arrival=float(t[i]), cfg=cfg))
    return reqs


def cell_count(cfg):
    nx, ny, nz = cfg["shape"]
    return nx * ny * nz


def state_bytes(cfg, bytes_per_value=4):
    """Bytes of one time level of all species (unpadded)."""
    return cell_count(cfg) * cfg["nspecies"] * bytes_per_value


def serving_mean_cells(edges=SERVE_EDGES):
    return float(np.mean([e ** 3 for e in edges]))



# --------------------------------------------------------------------------
# the same draws on a torch device (for large requests generated where they
# are used); bit patterns of uint64 arithmetic are carried in int64 tensors
# --------------------------------------------------------------------------
def _as_i64(u):
    u = int(u) & 0xFFFFFFFFFFFFFFFF
    return u - (1 << 64) if u >= (1 << 63) else u


def _lsr(z, k):
    """Logical right shift of int64 bit patterns."""
    return (z >> k) & ((1 << (64 - k)) - 1)


def uniform01_torch(seed, species, n, device, start=0):
    """``uniform01`` computed with torch on ``device`` (same values)."""
    import torch
    base = _as_i64((int(seed) * 0x9E3779B97F4A7C15) ^ (int(species) * 0xC2B2AE3D27D4EB4F))
    z = torch.arange(start, start + n, dtype=torch.int64, device=device) + base
    z = z + _as_i64(0x9E3779B97F4A7C15)
    z = (z ^ _lsr(z, 30)) * _as_i64(0xBF58476D1CE4E5B9)
    z = (z ^ _lsr(z, 27)) * _as_i64(0x94D049BB133111EB)
    z = z ^ _lsr(z, 31)
    return _lsr(z, 11).to(torch.float64) * (1.0 / 9007199254740992.0)


def initial_fields_torch(cfg, device, seed=None):
    """``initial_fields`` (float32) generated with torch on ``device``."""
    import torch
    nx, ny, nz = cfg["shape"]
    ncell = nx * ny * nz
    s = cfg["seed"] if seed is None else seed
    S = cfg["nspecies"]
    out = torch.empty((S, nz, ny, nx), dtype=torch.float64, device=device)
    kind = cfg["init"]
    if kind == "blob":
        u = uniform01_torch(s, 0, ncell, device).reshape(nz, ny, nx)
        z = torch.arange(nz, device=device, dtype=torch.float64).view(nz, 1, 1)
        y = torch.arange(ny, device=device, dtype=torch.float64).view(1, ny, 1)
        x = torch.arange(nx, device=device, dtype=torch.float64).view(1, 1, nx)
        cx, cy, cz = (nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0
        r2 = (x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2
        out[0] = u + 10.0 * torch.exp(-r2 / (2.0 * 6.0 ** 2))
    elif kind == "brusselator":
        a, b = cfg["params"]["a"], cfg["params"]["b"]
        base = (a, b / a)
        for sp in range(2):
            u = uniform01_torch(s, sp, ncell, device).reshape(nz, ny, nx)
            out[sp] = base[sp] * (1.0 + 0.01 * (2.0 * u - 1.0))
    elif kind == "ch_front":
        out[0] = 0.0
        out[0, 0, :, :] = cfg["bc_value"][0][4]
        out[1] = 1.0
        u = uniform01_torch(s, 2, ncell, device).reshape(nz, ny, nx)
        out[2] = 0.005 * (2.0 * u - 1.0)
    elif kind == "air":
        base = (0.01, 0.01, 1.0)
        for sp in range(3):
            u = uniform01_torch(s, sp, ncell, device).reshape(nz, ny, nx)
            out[sp] = base[sp] * (1.0 + 0.01 * (2.0 * u - 1.0))
    elif kind == "turing":
        sig = cfg["sigma"]
        for sp in range(2):
            u = uniform01_torch(s, sp, ncell, device).reshape(nz, ny, nx)
            out[sp] = 1.0 + sig * (2.0 * u - 1.0)
    elif kind == "zero":
        out[:] = 0.0
    elif kind == "ch_table1":
        out[0] = 0.0
        out[0, :, :, 0] = cfg["bc_value"][0][0]
        out[1] = 1.0
        out[2] = -1.0
    elif kind == "uniform_noise":
        for sp in range(S):
            out[sp] = uniform01_torch(s, sp, ncell, device).reshape(nz, ny, nx)
    else:
        raise ValueError(f"unknown initial condition {kind!r}")
    return out.to(torch.float32)
