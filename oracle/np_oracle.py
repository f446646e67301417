"""NumPy restatement of the forward-Euler method-of-lines step.

TEST INFRASTRUCTURE ONLY: an independent second oracle used to cross-check
the C stepper (``rd_oracle.c``).  It is written differently on purpose:
whole-array operations on a field padded by one ghost layer per axis
(``np.pad`` mode ``edge`` for zero-flux faces, ``wrap`` for periodic axes),
instead of per-cell boundary-aware accessors.

Definitions followed: eq. (1) with a diagonal D (per species and axis),
eq. (5) forward Euler, the 7-point Laplacian per axis or the 19-point
Laplacian of eqs. (3)-(4) (``cfg["stencil"] == 19``), first-order upwind
advection (Section 4.1), the Cahn-Hilliard biharmonic as Laplacian, boundary
rule, Laplacian (Section 4.1), held boundary layers for Dirichlet faces
(Section 4.1, boundary points set before each step).
"""
from __future__ import annotations

import numpy as np

# array axes are (z, y, x); face f -> array axis
_FACE_AXIS = {0: 2, 1: 2, 2: 1, 3: 1, 4: 0, 5: 0}


def _pad_axis(f, axis, periodic):
    widths = [(0, 0)] * f.ndim
    widths[axis] = (1, 1)
    return np.pad(f, widths, mode="wrap" if periodic else "edge")


def _shifted(f, axis, periodic):
    """(minus, plus) neighbour arrays of f along ``axis`` (array axis)."""
    g = _pad_axis(f, axis, periodic)
    n = f.shape[axis]
    lo = np.take(g, np.arange(0, n), axis=axis)
    hi = np.take(g, np.arange(2, n + 2), axis=axis)
    return lo, hi


def _periodic_axes(bc_s):
    # cfg axis a (0=x,1=y,2=z) -> periodic flag
    return [bc_s[2 * a] == "periodic" for a in range(3)]


def _second_diffs(f, bc_s, h):
    """Second differences along x, y, z (cfg axis order) divided by h^2."""
    per = _periodic_axes(bc_s)
    out = []
    for a, arr_axis in ((0, 2), (1, 1), (2, 0)):
        lo, hi = _shifted(f, arr_axis, per[a])
        out.append((lo + hi - 2.0 * f) / (h * h))
    return out


# eq. (4): T[r + 1][q + 1][p + 1] for offsets (p, q, r) along (x, y, z)
_T_PLUS = np.array([[0.0, 1.0, 0.0], [1.0, 2.0, 1.0], [0.0, 1.0, 0.0]])
_T_MID = np.array([[1.0, 2.0, 1.0], [2.0, -24.0, 2.0], [1.0, 2.0, 1.0]])
_T19 = np.stack([_T_PLUS, _T_MID, _T_PLUS])


def _lap19(f, bc_s, h):
    """Eq. (3): the 19-point Laplacian of f (nz, ny, nx).  The field is
    padded along x, then y, then z, so an edge ghost takes both crossed
    axes' rules in turn."""
    per = _periodic_axes(bc_s)
    g = f
    for a, arr_axis in ((0, 2), (1, 1), (2, 0)):
        g = _pad_axis(g, arr_axis, per[a])
    nz, ny, nx = f.shape
    acc = np.zeros_like(f)
    for r in range(3):
        for q in range(3):
            for p in range(3):
                w = _T19[r, q, p]
                if w:
                    acc += w * g[r:r + nz, q:q + ny, p:p + nx]
    return acc / (6.0 * h * h)


def _held_mask(shape, bc_s):
    """(face, index) pairs of the held (Dirichlet) layers of one species,
    faces in order -x,+x,-y,+y,-z,+z; where layers meet, the first face in
    that order gives the value (callers assign in reverse order)."""
    faces = []
    for f in range(6):
        if bc_s[f] != "dirichlet":
            continue
        axis = _FACE_AXIS[f]
        idx = [slice(None)] * 3
        idx[axis] = 0 if f % 2 == 0 else shape[axis] - 1
        faces.append((f, tuple(idx)))
    return faces


def _wind_profile(cfg):
    w = cfg.get("wind")
    nz = cfg["shape"][2]
    z = np.arange(nz, dtype=np.float64)
    if not w:
        return np.zeros(nz)
    if w["kind"] == "log":
        return w["u0"] * np.log1p(z) / np.log1p(float(nz))
    if w["kind"] == "const":
        return np.full(nz, float(w["u0"]))
    if w["kind"] == "table1":
        return np.zeros(nz)          # the three-axis wind is applied in np_step
    raise ValueError(w["kind"])


def _upwind(f, axis_cfg, u, bc_s, h):
    """-u d f / d(axis), first-order upwind (backward difference for u > 0)."""
    arr_axis = {0: 2, 1: 1, 2: 0}[axis_cfg]
    lo, hi = _shifted(f, arr_axis, _periodic_axes(bc_s)[axis_cfg])
    if u > 0:
        return -u * (f - lo) / h
    if u < 0:
        return -u * (hi - f) / h
    return np.zeros_like(f)


def _rates(cfg, c):
    """Reaction terms R(c) for all species, arrays of shape (nz, ny, nx)."""
    m = cfg["model"]
    P = cfg["params"]
    S = c.shape[0]
    r = [np.zeros_like(c[0]) for _ in range(S)]
    if m == "brusselator":
        u, v = c[0], c[1]
        uuv = u * u * v
        r[0] = P["a"] - (P["b"] + 1.0) * u + uuv
        r[1] = P["b"] * u - uuv
    elif m == "ch_front":
        q = P["k"] * c[0] * c[1]
        r[0], r[1], r[2] = -q, -q, q
    elif m == "air":
        photo = P["j"] * c[1]
        titr = P["k"] * c[0] * c[2]
        r[0] = photo - titr
        r[1] = titr - photo
        r[2] = photo - titr
    elif m == "ch_table1":
        c1, c2, c3 = c[0], c[1], c[2]
        q = P["k1"] * c1 * c2
        sink = P["k2"] * c1 * c3
        r[0] = -q - sink
        r[1] = -q
        r[2] = q - sink
    elif m == "turing":
        c1, c2 = c[0], c[1]
        r[0] = c1 - c1 ** 3 - c2
        r[1] = P["gamma"] * (c1 - P["alpha"] * c2 - P["beta"])
    return r


def np_step(cfg, c, n=0):
    """Step number ``n`` (time n dt at its start); c has shape
    (S, nz, ny, nx) float64; returns the new array."""
    S = cfg["nspecies"]
    h, dt = cfg["h"], cfg["dt"]
    stencil = cfg.get("stencil", 7)
    if stencil not in (7, 19):
        raise ValueError(f"stencil {stencil}")
    if stencil == 19 and any(len(set(d)) != 1 for d in cfg["D"][:S]):
        raise ValueError("eq. (3) has one diffusivity per species")
    c = c.copy()
    held = [_held_mask(c.shape[1:], cfg["bc"][s]) for s in range(S)]
    for s in range(S):
        for f, idx in reversed(held[s]):
            c[s][idx] = cfg["bc_value"][s][f]
    rates = _rates(cfg, c)
    u = _wind_profile(cfg)[:, None, None]
    out = np.empty_like(c)
    for s in range(S):
        bc_s = cfg["bc"][s]
        D = cfg["D"][s]
        if stencil == 19:
            lap_c = _lap19(c[s], bc_s, h)
            tend = rates[s] + D[0] * lap_c
        else:
            dxx, dyy, dzz = _second_diffs(c[s], bc_s, h)
            lap_c = dxx + dyy + dzz
            tend = rates[s] + D[0] * dxx + D[1] * dyy + D[2] * dzz
        w = cfg.get("wind")
        if w and w["kind"] == "table1":
            u3 = (w["ux"], w["uy"], w["uz_amp"] * np.sin(n * dt / w["uz_tau"]))
            for a in range(3):
                tend = tend + _upwind(c[s], a, u3[a], bc_s, h)
        elif w:
            per_x = bc_s[0] == "periodic"
            xm, xp = _shifted(c[s], 2, per_x)
            back = (c[s] - xm) / h
            fwd = (xp - c[s]) / h
            tend = tend - np.where(u > 0, u * back, u * fwd)
        if cfg["model"] == "ch_front" and s == 2:
            P = cfg["params"]
            cc = c[2]
            mu = 2.0 * cc * (cc - 1.0) * (2.0 * cc - 1.0) - P["kappa"] * lap_c
            if stencil == 19:
                lap_mu = _lap19(mu, bc_s, h)
            else:
                mx, my, mz = _second_diffs(mu, bc_s, h)
                lap_mu = mx + my + mz
            tend = tend + P["M"] * lap_mu
        if cfg["model"] == "ch_table1" and s == 2:
            P = cfg["params"]
            cc = c[2]
            lap_c = _lap19(cc, bc_s, h) if stencil == 19 else sum(_second_diffs(cc, bc_s, h))
            bracket = P["eps"] * cc - P["gamma"] * cc ** 3 + P["sigma"] * lap_c
            lap_b = (_lap19(bracket, bc_s, h) if stencil == 19
                     else sum(_second_diffs(bracket, bc_s, h)))
            tend = tend - P["lam"] * lap_b
        src = cfg.get("source")
        if src and src["species"] == s:
            tend[src["z"], src["y"], src["x"]] += src["rate"]
        out[s] = c[s] + dt * tend
        for f, idx in reversed(held[s]):
            out[s][idx] = cfg["bc_value"][s][f]
    return out


def np_run(cfg, fields, nsteps, n0=0):
    """Advance ``fields`` (S, nz, ny, nx) by ``nsteps`` steps in float64, the
    first step having index ``n0``."""
    c = np.asarray(fields, dtype=np.float64).copy()
    for k in range(int(nsteps)):
        c = np_step(cfg, c, n0 + k)
    return c
