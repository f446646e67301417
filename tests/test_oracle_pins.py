"""Pins of the FP64 oracle to facts that do not come from the oracle itself.

Each test checks the oracle against a closed form, an exact invariant, a
special case that reduces to a textbook result, or an independent matrix
construction, chosen so that a plausible slip (dropped term, wrong sign,
wrong index, transposed axis, wrong boundary rule) breaks at least one.

Definitions pinned: eq. (1)/(2) diffusion with diagonal D, the 7-point
Laplacian, the 19-point Laplacian of eqs. (3)-(4), eq. (5) forward Euler, first-order upwind advection and the
Cahn-Hilliard chained Laplacian of Section 4.1, boundary layers of
Section 4.1, and the reaction terms of the benchmark problems.
"""
import math

import numpy as np
import pytest

from paper_1004_0480_gb300 import workloads as W


def _diff_cfg(shape, D=(1.0, 1.0, 1.0), dt=0.05, bc="neumann", h=1.0):
    cfg = W.diffusion_blob(shape=shape, dt=dt, h=h)
    cfg["D"] = [list(D)]
    cfg["bc"] = [[bc] * 6]
    return cfg


# --------------------------------------------------------------------------
# Laplacian + Euler: Fourier modes decay by the exact discrete symbol
# --------------------------------------------------------------------------
@pytest.mark.parametrize("impl", ["c", "np"])
def test_fourier_mode_periodic(orc, impl):
    nx, ny, nz = 16, 12, 10
    m = (2, 1, 3)
    D = (1.0, 0.5, 0.25)
    h, dt = 0.7, 0.05
    cfg = _diff_cfg((nx, ny, nz), D=D, dt=dt, bc="periodic", h=h)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    mode = (np.cos(2 * np.pi * m[0] * x / nx) * np.cos(2 * np.pi * m[1] * y / ny)
            * np.cos(2 * np.pi * m[2] * z / nz))
    c0 = (1.0 + mode)[None]
    n = 25
    g = 1.0 - 4.0 * sum(D[d] * dt / h ** 2 * math.sin(math.pi * m[d] / N) ** 2
                        for d, N in enumerate((nx, ny, nz)))
    run = orc.run if impl == "c" else orc.np_run
    out = run(cfg, c0, n)[0]
    np.testing.assert_allclose(out, 1.0 + g ** n * mode, rtol=0, atol=1e-12)


@pytest.mark.parametrize("impl", ["c", "np"])
def test_fourier_mode_neumann(orc, impl):
    # cell-centred zero-flux eigenmodes cos(pi m (i + 1/2) / n)
    nx, ny, nz = 9, 14, 11
    m = (1, 3, 2)
    D = (0.3, 1.0, 0.6)
    dt = 0.08
    cfg = _diff_cfg((nx, ny, nz), D=D, dt=dt, bc="neumann")
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    mode = (np.cos(np.pi * m[0] * (x + 0.5) / nx) * np.cos(np.pi * m[1] * (y + 0.5) / ny)
            * np.cos(np.pi * m[2] * (z + 0.5) / nz))
    n = 30
    g = 1.0 - 4.0 * sum(D[d] * dt * math.sin(math.pi * m[d] / (2 * N)) ** 2
                        for d, N in enumerate((nx, ny, nz)))
    run = orc.run if impl == "c" else orc.np_run
    out = run(cfg, (2.0 + mode)[None], n)[0]
    np.testing.assert_allclose(out, 2.0 + g ** n * mode, rtol=0, atol=1e-12)


def test_stability_bound_checkerboard(orc):
    # the checkerboard is the fastest mode: g = 1 - 12 r with r = D dt / h^2;
    # it stays bounded iff dt <= h^2 / (6 D)
    n = 8
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    cb = ((-1.0) ** (x + y + z))[None]
    for factor, grows in ((1.0 + 1e-2, True), (1.0 - 1e-2, False)):
        dt = factor / 6.0
        cfg = _diff_cfg((n, n, n), dt=dt, bc="periodic")
        out = orc.run(cfg, cb, 200)
        g = 1.0 - 12.0 * dt
        np.testing.assert_allclose(out, g ** 200 * cb, rtol=1e-10, atol=0)
        assert (np.abs(out).max() > 1.0) == grows


@pytest.mark.parametrize("bc", ["neumann", "periodic"])
def test_mass_conserved_pure_diffusion(orc, bc):
    cfg = _diff_cfg((10, 7, 9), D=(1.0, 0.4, 0.7), dt=0.1, bc=bc)
    c0 = W.initial_fields(W.with_(cfg, init="uniform_noise"), seed=11).astype(np.float64)
    out = orc.run(cfg, c0, 40)
    assert abs(out.sum() - c0.sum()) <= 1e-12 * abs(c0.sum())
    assert not np.allclose(out, c0)


# --------------------------------------------------------------------------
# independent matrix construction on a tiny grid (Kronecker sums)
# --------------------------------------------------------------------------
def _lap1d(n, periodic):
    A = -2.0 * np.eye(n) + np.eye(n, k=1) + np.eye(n, k=-1)
    if periodic:
        A[0, -1] = A[-1, 0] = 1.0
    else:
        A[0, 0] = A[-1, -1] = -1.0   # zero flux: ghost equals the face cell
    return A


def _upwind1d(n, periodic):
    # -(c_i - c_{i-1}) for positive velocity
    B = -np.eye(n) + np.eye(n, k=-1)
    if periodic:
        B[0, -1] = 1.0
    else:
        B[0, 0] = 0.0                # zero-gradient inflow
    return B


@pytest.mark.parametrize("bc", ["neumann", "periodic"])
def test_dense_operator_power(orc, bc):
    nx, ny, nz = 3, 4, 5
    per = bc == "periodic"
    D = (0.3, 0.2, 0.1)
    h, dt, u = 1.0, 0.2, 0.8
    cfg = _diff_cfg((nx, ny, nz), D=D, dt=dt, bc=bc, h=h)
    cfg["wind"] = dict(kind="const", u0=u)
    Ix, Iy, Iz = np.eye(nx), np.eye(ny), np.eye(nz)
    # array index order (z, y, x) -> kron(z, y, x)
    A = (D[0] * np.kron(Iz, np.kron(Iy, _lap1d(nx, per)))
         + D[1] * np.kron(Iz, np.kron(_lap1d(ny, per), Ix))
         + D[2] * np.kron(_lap1d(nz, per), np.kron(Iy, Ix))) / h ** 2
    A += u / h * np.kron(Iz, np.kron(Iy, _upwind1d(nx, per)))
    step = np.eye(nx * ny * nz) + dt * A
    c0 = W.uniform01(5, 0, nx * ny * nz)
    n = 17
    ref = np.linalg.matrix_power(step, n) @ c0
    out = orc.run(cfg, c0.reshape(1, nz, ny, nx), n).ravel()
    np.testing.assert_allclose(out, ref, rtol=0, atol=1e-13)


def _three_point_1d(p, r, bc, n):
    """The textbook explicit scheme u_i <- u_i + r (u_{i-1} - 2 u_i + u_{i+1}),
    zero flux (u_{-1} = u_0, u_N = u_{N-1}) or periodic, n steps."""
    u = [float(v) for v in p]
    N = len(u)
    for _ in range(n):
        new = []
        for i in range(N):
            if bc == "periodic":
                lo, hi = u[(i - 1) % N], u[(i + 1) % N]
            else:
                lo, hi = u[max(i - 1, 0)], u[min(i + 1, N - 1)]
            new.append(u[i] + r * (lo - 2.0 * u[i] + hi))
        u = new
    return np.array(u)


@pytest.mark.parametrize("impl", ["c", "np"])
@pytest.mark.parametrize("bc", ["neumann", "periodic"])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_one_axis_profile_reduces_to_the_three_point_scheme(orc, impl, bc, axis):
    # a field that varies along one axis only: the other axes' second
    # differences vanish, and the 3-D step is the 1-D scheme with that
    # axis's own D (every axis has a different one, so a D taken from the
    # wrong axis, or a profile moved along the wrong axis, fails)
    shape = (11, 7, 9)                       # (nx, ny, nz)
    D = (0.9, 0.4, 0.15)
    h, dt = 0.8, 0.1
    cfg = _diff_cfg(shape, D=D, dt=dt, bc=bc, h=h)
    N = shape[axis]
    prof = np.random.default_rng(7 + axis).uniform(0.0, 2.0, N)
    bshape = [1, 1, 1]
    bshape[2 - axis] = N                     # arrays are (z, y, x)
    c0 = np.broadcast_to(prof.reshape(bshape), shape[::-1]).copy()[None]
    n = 20
    want = _three_point_1d(prof, D[axis] * dt / h ** 2, bc, n)
    run = orc.run if impl == "c" else orc.np_run
    out = run(cfg, c0, n)[0]
    np.testing.assert_allclose(out, np.broadcast_to(want.reshape(bshape), out.shape),
                               rtol=0, atol=1e-13)


# --------------------------------------------------------------------------
# advection
# --------------------------------------------------------------------------
def test_upwind_courant_one_is_exact_shift(orc):
    nx, ny, nz = 12, 3, 4
    h, dt = 1.0, 0.25
    cfg = _diff_cfg((nx, ny, nz), D=(0, 0, 0), dt=dt, bc="periodic", h=h)
    cfg["wind"] = dict(kind="const", u0=h / dt)
    c0 = W.uniform01(9, 0, nx * ny * nz).reshape(1, nz, ny, nx)
    n = 5
    out = orc.run(cfg, c0, n)
    np.testing.assert_allclose(out, np.roll(c0, n, axis=3), rtol=0, atol=1e-15)


def test_log_wind_profile_on_linear_field(orc):
    # c = alpha x + beta, no diffusion: away from the inflow face the update
    # is c - dt u(z) alpha / h with u(z) = ln(1+z)/ln(1+nz), z the cell index;
    # at x = 0 the zero-gradient ghost gives no change
    nx, ny, nz = 6, 2, 7
    alpha, beta, dt, h = 0.5, 2.0, 0.1, 1.0
    cfg = _diff_cfg((nx, ny, nz), D=(0, 0, 0), dt=dt, bc="neumann", h=h)
    cfg["wind"] = dict(kind="log", u0=1.0)
    x = np.arange(nx)[None, None, :] * np.ones((nz, ny, 1))
    c0 = (alpha * x + beta)[None]
    out = orc.run(cfg, c0, 1)[0]
    uz = np.log(1.0 + np.arange(nz)) / np.log(1.0 + nz)
    expect = c0[0] - dt * uz[:, None, None] * alpha / h
    expect[:, :, 0] = c0[0][:, :, 0]
    np.testing.assert_allclose(out, expect, rtol=0, atol=1e-14)


def test_log_wind_budget_telescopes(orc):
    # sum over x of the upwind term telescopes to -u (c_{n-1} - c_0) / h
    cfg = W.air((10, 6, 8), src=(1, 1, 1), src_rate=0.0, j=0.0, k=0.0)
    c0 = W.initial_fields(W.with_(cfg, init="uniform_noise"), seed=3).astype(np.float64)
    c1 = orc.run(cfg, c0, 1)
    uz = np.log1p(np.arange(8.0)) / np.log1p(8.0)
    for s in range(3):
        flux = (uz[:, None] * (c0[s, :, :, -1] - c0[s, :, :, 0])).sum()
        assert abs((c1[s].sum() - c0[s].sum()) - (-cfg["dt"] * flux)) < 1e-12


# --------------------------------------------------------------------------
# reactions
# --------------------------------------------------------------------------
def test_brusselator_steady_state_bitwise(orc):
    cfg = W.brusselator(shape=(6, 5, 4), bc="periodic")
    c0 = np.empty((2, 4, 5, 6))
    c0[0], c0[1] = 3.0, 3.0     # (a, b/a) with a = 3, b = 9
    out = orc.run(cfg, c0, 50)
    assert np.array_equal(out, c0)


def test_brusselator_sum_identity(orc):
    # f + g = a - u for the Brusselator, so for a uniform state
    # (u + v)_{n+1} = (u + v)_n + dt (a - u_n), whatever u^2 v is
    cfg = W.brusselator(shape=(4, 4, 4))
    c0 = np.empty((2, 4, 4, 4))
    c0[0], c0[1] = 1.3, 2.1
    c1 = orc.run(cfg, c0, 1)
    assert np.ptp(c1[0]) == 0 and np.ptp(c1[1]) == 0
    lhs = c1[0, 0, 0, 0] + c1[1, 0, 0, 0]
    rhs = 1.3 + 2.1 + cfg["dt"] * (3.0 - 1.3)
    assert abs(lhs - rhs) < 1e-14


def test_brusselator_linearised_mode(orc):
    # small periodic mode about (a, b/a): per step the amplitudes follow
    # I + dt (J - lam diag(Du, Dv)), J = [[b-1, a^2], [-b, -a^2]] (textbook
    # Brusselator Jacobian), lam = 4 sin^2(pi m / n) / h^2
    a, b, Du, Dv, dt, n = 3.0, 9.0, 2.0, 16.0, 0.005, 16
    cfg = W.brusselator(shape=(n, 4, 4), a=a, b=b, Du=Du, Dv=Dv, dt=dt)
    m = 2
    x = np.arange(n)
    mode = np.cos(2 * np.pi * m * x / n)[None, None, :] * np.ones((4, 4, 1))
    eps = np.array([1e-7, -2e-7])
    c0 = np.stack([a + eps[0] * mode, b / a + eps[1] * mode])
    steps = 60
    out = orc.run(cfg, c0, steps)
    lam = 4.0 * math.sin(math.pi * m / n) ** 2
    J = np.array([[b - 1.0, a * a], [-b, -a * a]]) - lam * np.diag([Du, Dv])
    amp = np.linalg.matrix_power(np.eye(2) + dt * J, steps) @ eps
    got = np.array([(out[0] - a)[0, 0, 0], (out[1] - b / a)[0, 0, 0]])
    np.testing.assert_allclose(got, amp, rtol=2e-5)


@pytest.mark.parametrize("stencil", [7, 19])
def test_turing_linearised_mode(orc, stencil):
    # small x-y mode about the homogeneous steady state of the Table 1
    # activator-inhibitor system: per step the amplitudes follow
    # I + dt (J - lam diag(D1, D2)) with the textbook Jacobian
    # J = [[1 - 3 c1^2, -1], [gamma, -gamma alpha]] and lam the stencil's
    # symbol (7-point: sum of 4 sin^2(theta/2) / h^2; 19-point: eq. (3)'s)
    n = 12
    cfg = W.turing(shape=(n, n, 3), stencil=stencil)
    cfg["bc"] = [["periodic"] * 6] * 2
    al, be, ga = (cfg["params"][k] for k in ("alpha", "beta", "gamma"))
    D1, D2 = cfg["D"][0][0], cfg["D"][1][0]
    h, dt = cfg["h"], cfg["dt"]
    # steady state: c2 = (c1 - beta) / alpha and c1 - c1^3 - c2 = 0
    roots = np.roots([1.0, 0.0, 1.0 / al - 1.0, -be / al])
    c1 = float(roots[np.abs(roots.imag) < 1e-12].real[0])
    c2 = (c1 - be) / al
    mx, my = 2, 1
    z, y, x = np.meshgrid(np.arange(3), np.arange(n), np.arange(n), indexing="ij")
    th = (2 * np.pi * mx / n, 2 * np.pi * my / n)
    mode = np.cos(th[0] * x + th[1] * y)
    eps = np.array([1e-7, -3e-7])
    c0 = np.stack([c1 + eps[0] * mode, c2 + eps[1] * mode])
    steps = 40
    out = orc.run(cfg, c0, steps)
    if stencil == 7:
        lam = sum(4.0 * math.sin(t / 2) ** 2 for t in th) / h ** 2
    else:
        lam = -_symbol19((th[0], th[1], 0.0)) / (6.0 * h ** 2)
    J = np.array([[1.0 - 3.0 * c1 * c1, -1.0], [ga, -ga * al]]) - lam * np.diag([D1, D2])
    amp = np.linalg.matrix_power(np.eye(2) + dt * J, steps) @ eps
    got = np.array([(out[0] - c1)[0, 0, 0], (out[1] - c2)[0, 0, 0]])
    np.testing.assert_allclose(got, amp, rtol=2e-5)


def test_air_photostationary_state_bitwise(orc):
    # j NO2 = k NO O3 is a steady state of NO2 <-> NO + O3
    cfg = W.air((5, 4, 3), src=(0, 0, 0), src_rate=0.0, j=0.5, k=2.0)
    cfg["wind"] = None
    c0 = np.empty((3, 3, 4, 5))
    c0[0], c0[1], c0[2] = 1.0, 4.0, 1.0     # NO, NO2, O3
    out = orc.run(cfg, c0, 20)
    assert np.array_equal(out, c0)


def test_air_first_order_photolysis(orc):
    # with k = 0, NO2 decays as (1 - j dt)^n, NO and O3 gain what it loses
    cfg = W.air((4, 4, 4), src=(0, 0, 0), src_rate=0.0, j=0.5, k=0.0)
    cfg["wind"] = None
    c0 = np.zeros((3, 4, 4, 4))
    c0[1] = 1.0
    n = 7
    out = orc.run(cfg, c0, n)
    nd = (1.0 - 0.5 * cfg["dt"]) ** n
    np.testing.assert_allclose(out[1], nd, rtol=1e-14)
    np.testing.assert_allclose(out[0], 1.0 - nd, rtol=1e-13)
    np.testing.assert_allclose(out[2], 1.0 - nd, rtol=1e-13)


def test_air_budgets_and_source_position(orc):
    cfg = W.air((9, 7, 6), src=(2, 5, 3), src_rate=1.0)
    cfg["wind"] = None
    c0 = W.initial_fields(cfg).astype(np.float64)
    n = 6
    out = orc.run(cfg, c0, n)
    tot = lambda a: a.sum()
    # NO2 + O3 is conserved; NO + NO2 grows by dt * rate per step
    assert abs(tot(out[1] + out[2]) - tot(c0[1] + c0[2])) < 1e-11
    assert abs(tot(out[0] + out[1]) - tot(c0[0] + c0[1]) - n * cfg["dt"]) < 1e-11
    # the emission lands at (x, y, z) = (2, 5, 3)
    z0 = np.zeros_like(c0)
    one = orc.run(cfg, z0, 1)
    assert np.unravel_index(np.argmax(one[0]), one[0].shape) == (3, 5, 2)
    assert one[0].sum() == pytest.approx(cfg["dt"], abs=1e-15)


def test_front_reaction_invariants(orc):
    # a + b -> c: a - b and a + c are conserved; one step of a uniform state
    # removes dt k a b from a and b
    cfg = W.ch_front(shape=(5, 5, 5))
    cfg["bc"] = [["neumann"] * 6 for _ in range(3)]
    c0 = np.empty((3, 5, 5, 5))
    c0[0], c0[1], c0[2] = 0.7, 1.4, 0.25
    out = orc.run(cfg, c0, 10)
    assert np.ptp(out) < 1e-15 or all(np.ptp(out[s]) == 0 for s in range(3))
    np.testing.assert_allclose(out[0] - out[1], 0.7 - 1.4, rtol=0, atol=1e-14)
    np.testing.assert_allclose(out[0] + out[2], 0.95, rtol=0, atol=1e-14)
    one = orc.run(cfg, c0, 1)
    np.testing.assert_allclose(one[0], 0.7 - cfg["dt"] * 0.7 * 1.4, rtol=1e-15)


@pytest.mark.parametrize("cbar,fprime", [(0.0, 2.0), (0.5, -1.0)])
def test_cahn_hilliard_linear_symbol(orc, cbar, fprime):
    # about a uniform c, a small mode evolves by
    # 1 - dt M lam (kappa lam + f''(cbar)),  f'(c) = 2c(c-1)(2c-1)
    n, dt, M, kappa = 12, 0.01, 0.1, 1.0
    cfg = W.ch_front(shape=(n, n, 4), dt=dt, M=M, kappa=kappa, k=0.0, Da=0.0, Db=0.0)
    cfg["bc"] = [["periodic"] * 6 for _ in range(3)]
    cfg["bc_value"] = [[0.0] * 6 for _ in range(3)]
    mx, my = 1, 2
    z, y, x = np.meshgrid(np.arange(4), np.arange(n), np.arange(n), indexing="ij")
    mode = np.cos(2 * np.pi * mx * x / n) * np.cos(2 * np.pi * my * y / n)
    eps = 1e-7
    c0 = np.zeros((3, 4, n, n))
    c0[2] = cbar + eps * mode
    steps = 40
    out = orc.run(cfg, c0, steps)
    lam = 4.0 * (math.sin(math.pi * mx / n) ** 2 + math.sin(math.pi * my / n) ** 2)
    g = 1.0 - dt * M * lam * (kappa * lam + fprime)
    np.testing.assert_allclose(out[2] - cbar, g ** steps * eps * mode, rtol=0,
                               atol=1e-5 * eps)


def test_cahn_hilliard_mass_conserved_neumann(orc):
    cfg = W.ch_front(shape=(8, 7, 6), k=0.0)
    cfg["bc"] = [["neumann"] * 6 for _ in range(3)]
    c0 = W.initial_fields(cfg).astype(np.float64)
    c0[2] += 0.3
    out = orc.run(cfg, c0, 50)
    assert abs(out[2].sum() - c0[2].sum()) < 1e-12 * c0[2].size
    assert not np.allclose(out[2], c0[2])


# --------------------------------------------------------------------------
# held (Dirichlet) boundary layers
# --------------------------------------------------------------------------
def test_dirichlet_linear_profile_is_steady(orc):
    # held layers at z = 0 (value 10) and z = nz-1 (value 0): the linear
    # profile through the cell planes has zero second difference
    nz = 9
    cfg = _diff_cfg((5, 4, nz), dt=0.1, bc="neumann")
    cfg["bc"][0][4] = cfg["bc"][0][5] = "dirichlet"
    cfg["bc_value"] = [[0, 0, 0, 0, 10.0, 0.0]]
    prof = 10.0 * (1.0 - np.arange(nz) / (nz - 1))
    c0 = (prof[:, None, None] * np.ones((nz, 4, 5)))[None]
    out = orc.run(cfg, c0, 30)
    np.testing.assert_allclose(out, c0, rtol=0, atol=1e-12)
    # a zero start relaxes towards that profile, the layers held throughout
    out = orc.run(cfg, np.zeros_like(c0), 3000)
    assert np.all(out[0, 0] == 10.0) and np.all(out[0, -1] == 0.0)
    np.testing.assert_allclose(out, c0, rtol=0, atol=1e-6)


@pytest.mark.parametrize("model", ["brusselator", "air", "ch_front", "turing", "ch_table1"])
def test_uniform_state_follows_the_scalar_ode(orc, model):
    # with every face periodic and no wind or source, a uniform state stays
    # uniform and each cell follows the forward-Euler map of the model's
    # ODE, written here from the kinetics of the benchmark problems
    if model == "brusselator":
        cfg = W.brusselator(shape=(5, 4, 6))
        y0 = [1.0, 2.0]
        a, b = cfg["params"]["a"], cfg["params"]["b"]

        def rate(y):
            u, v = y
            return [a - (b + 1.0) * u + u * u * v, b * u - u * u * v]
    elif model == "air":
        cfg = W.air((5, 4, 6), src=(0, 0, 0))
        cfg["source"], cfg["wind"] = None, None
        y0 = [0.2, 0.5, 0.8]
        j, k = cfg["params"]["j"], cfg["params"]["k"]

        def rate(y):
            no, no2, o3 = y
            net = j * no2 - k * no * o3          # NO2 -> NO + O3 minus NO + O3 -> NO2
            return [net, -net, net]
    elif model == "turing":
        cfg = W.turing(shape=(5, 4, 6))
        y0 = [0.7, 0.4]
        al, be, ga = (cfg["params"][k] for k in ("alpha", "beta", "gamma"))

        def rate(y):
            # activator-inhibitor kinetics of Table 1, row 2
            return [y[0] - y[0] ** 3 - y[1], ga * (y[0] - al * y[1] - be)]
    elif model == "ch_table1":
        cfg = W.ch_table1(shape=(5, 4, 6), k2=0.05)
        y0 = [0.9, 0.6, -0.4]
        k1, k2 = cfg["params"]["k1"], cfg["params"]["k2"]

        def rate(y):
            # Table 1, row 3: c1 + c2 -> c3 and the sink k2 c1 c3; the
            # Cahn-Hilliard term vanishes on a uniform state
            q, sink = k1 * y[0] * y[1], k2 * y[0] * y[2]
            return [-q - sink, -q, q - sink]
    else:
        cfg = W.ch_front(shape=(5, 4, 6))
        y0 = [0.9, 0.6, 0.3]
        k = cfg["params"]["k"]

        def rate(y):
            q = k * y[0] * y[1]                  # a + b -> c; mu is uniform
            return [-q, -q, q]
    S = cfg["nspecies"]
    cfg["bc"] = [["periodic"] * 6 for _ in range(S)]
    cfg["bc_value"] = [[0.0] * 6 for _ in range(S)]
    c0 = np.stack([np.full((6, 4, 5), v) for v in y0])
    steps = 25
    out = orc.run(cfg, c0, steps)
    y = list(y0)
    for _ in range(steps):
        r = rate(y)
        y = [y[s] + cfg["dt"] * r[s] for s in range(S)]
    for s in range(S):
        assert np.ptp(out[s]) == 0.0
        assert out[s].flat[0] == pytest.approx(y[s], rel=1e-13, abs=1e-15)
    assert any(abs(y[s] - y0[s]) > 1e-3 for s in range(S))   # the state moved


def test_mirror_ghost_equivalence_for_cahn_hilliard(orc):
    # Section 4.1 re-applies the boundary rule to mu before the second
    # Laplacian.  At zero-flux faces that equals extending c by two mirrored
    # cells (ghost(-1) = c(0), ghost(-2) = c(1)) and evaluating mu on the
    # ghosts: computed here with np.pad, against one oracle step
    shape = (7, 6, 5)
    cfg = W.ch_front(shape=shape, k=0.0, Da=0.0, Db=0.0)
    cfg["bc"] = [["neumann"] * 6 for _ in range(3)]
    cfg["bc_value"] = [[0.0] * 6 for _ in range(3)]
    rng = np.random.default_rng(7)
    c0 = np.zeros((3, 5, 6, 7))
    c0[2] = 0.5 + 0.3 * rng.standard_normal((5, 6, 7))
    out = orc.run(cfg, c0, 1)
    h2 = cfg["h"] ** 2
    kappa, M, dt = cfg["params"]["kappa"], cfg["params"]["M"], cfg["dt"]
    c = np.pad(c0[2], 2, mode="symmetric")            # (z, y, x), two ghost layers

    def lap(f):   # 7-point Laplacian on the interior one cell in from f's edge
        return (f[2:, 1:-1, 1:-1] + f[:-2, 1:-1, 1:-1] + f[1:-1, 2:, 1:-1] + f[1:-1, :-2, 1:-1]
                + f[1:-1, 1:-1, 2:] + f[1:-1, 1:-1, :-2] - 6.0 * f[1:-1, 1:-1, 1:-1]) / h2
    cm = c[1:-1, 1:-1, 1:-1]                          # the grid plus one ghost layer
    mu = 2.0 * cm * (cm - 1.0) * (2.0 * cm - 1.0) - kappa * lap(c)
    expect = c0[2] + dt * M * lap(mu)
    np.testing.assert_allclose(out[2], expect, rtol=0, atol=1e-13)
    np.testing.assert_array_equal(out[0], c0[0])


# --------------------------------------------------------------------------
# the 19-point Laplacian of eqs. (3)-(4)
# --------------------------------------------------------------------------
def _symbol19(theta):
    """(6 h^2) times the eigenvalue of eq. (3) on exp(i theta . x): face
    neighbours (weight 2) give 4 cos(theta_d), the four edge neighbours of
    each axis pair (weight 1) give 4 cos(theta_d) cos(theta_e)."""
    c = [math.cos(t) for t in theta]
    return -24.0 + 4.0 * sum(c) + 4.0 * (c[0] * c[1] + c[0] * c[2] + c[1] * c[2])


def _cfg19(shape, D=1.0, dt=0.05, bc="neumann", h=1.0):
    cfg = _diff_cfg(shape, D=(D, D, D), dt=dt, bc=bc, h=h)
    cfg["stencil"] = 19
    return cfg


@pytest.mark.parametrize("impl", ["c", "np"])
def test_stencil19_oblique_plane_wave_periodic(orc, impl):
    # cos(theta . x) with all three wave numbers non-zero: the edge weights
    # enter through the products cos(theta_d) cos(theta_e)
    nx, ny, nz = 12, 10, 8
    m = (1, 3, 2)
    D, h, dt = 0.8, 0.7, 0.06
    cfg = _cfg19((nx, ny, nz), D=D, dt=dt, bc="periodic", h=h)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    theta = [2 * np.pi * m[d] / N for d, N in enumerate((nx, ny, nz))]
    mode = np.cos(theta[0] * x + theta[1] * y + theta[2] * z)
    g = 1.0 + D * dt / (6.0 * h * h) * _symbol19(theta)
    n = 20
    run = orc.run if impl == "c" else orc.np_run
    out = run(cfg, (1.0 + mode)[None], n)[0]
    np.testing.assert_allclose(out, 1.0 + g ** n * mode, rtol=0, atol=1e-12)


@pytest.mark.parametrize("impl", ["c", "np"])
def test_stencil19_cosine_mode_neumann(orc, impl):
    # cell-centred zero-flux modes: each axis's reflecting shift-sum has
    # eigenvalue 2 cos(pi m / n), and the edge ghosts compose the face rules,
    # so the product mode keeps the symbol at theta_d = pi m_d / n_d
    nx, ny, nz = 9, 7, 8
    m = (2, 1, 3)
    D, dt = 0.5, 0.1
    cfg = _cfg19((nx, ny, nz), D=D, dt=dt, bc="neumann")
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    mode = (np.cos(np.pi * m[0] * (x + 0.5) / nx) * np.cos(np.pi * m[1] * (y + 0.5) / ny)
            * np.cos(np.pi * m[2] * (z + 0.5) / nz))
    theta = [np.pi * m[d] / N for d, N in enumerate((nx, ny, nz))]
    g = 1.0 + D * dt / 6.0 * _symbol19(theta)
    n = 25
    run = orc.run if impl == "c" else orc.np_run
    out = run(cfg, (3.0 + mode)[None], n)[0]
    np.testing.assert_allclose(out, 3.0 + g ** n * mode, rtol=0, atol=1e-12)


def _shift_sum1d(n, periodic):
    # c[i-1] + c[i+1] with the face rule of the axis
    return _lap1d(n, periodic) + 2.0 * np.eye(n)


@pytest.mark.parametrize("per", [(True, True, True), (False, False, False),
                                 (True, False, False), (False, True, False)])
def test_stencil19_dense_operator_power(orc, per):
    # eq. (3) as a matrix: -24 I + 2 (Sx + Sy + Sz) + Sx Sy + Sx Sz + Sy Sz
    # over 6 h^2, S_a the shift-sum of axis a; mixed boundary rules check that
    # an edge ghost takes each crossed axis's own rule
    nx, ny, nz = 4, 3, 5
    D, h, dt, u = 0.3, 0.9, 0.2, 0.5
    cfg = _cfg19((nx, ny, nz), D=D, dt=dt, h=h)
    cfg["bc"] = [[("periodic" if per[f // 2] else "neumann") for f in range(6)]]
    cfg["wind"] = dict(kind="const", u0=u)
    Ix, Iy, Iz = np.eye(nx), np.eye(ny), np.eye(nz)
    Sx = np.kron(Iz, np.kron(Iy, _shift_sum1d(nx, per[0])))
    Sy = np.kron(Iz, np.kron(_shift_sum1d(ny, per[1]), Ix))
    Sz = np.kron(_shift_sum1d(nz, per[2]), np.kron(Iy, Ix))
    N = nx * ny * nz
    L = (-24.0 * np.eye(N) + 2.0 * (Sx + Sy + Sz) + Sx @ Sy + Sx @ Sz + Sy @ Sz) / (6 * h * h)
    A = D * L + u / h * np.kron(Iz, np.kron(Iy, _upwind1d(nx, per[0])))
    step = np.eye(N) + dt * A
    c0 = W.uniform01(9, 0, N)
    n = 11
    ref = np.linalg.matrix_power(step, n) @ c0
    out = orc.run(cfg, c0.reshape(1, nz, ny, nx), n).ravel()
    np.testing.assert_allclose(out, ref, rtol=0, atol=1e-13)


def test_stencil19_exact_on_cubic_polynomials(orc):
    # both stencils are exact for polynomials of degree <= 3 (the weights of
    # eq. (4) are even in each offset and sum p^2 T_pqr = 12 per axis); away
    # from the faces one step adds dt D times the analytic Laplacian
    nx, ny, nz = 9, 8, 7
    h, D, dt = 0.5, 0.7, 0.01
    z, y, x = np.meshgrid(np.arange(nz) * h, np.arange(ny) * h, np.arange(nx) * h,
                          indexing="ij")
    c = (1.0 + 0.3 * x - 0.2 * y + 0.1 * z + 0.05 * x * x + 0.02 * x * y - 0.03 * y * y
         + 0.04 * y * z + 0.01 * z * z + 0.002 * x ** 3 - 0.001 * x * y * z + 0.003 * z ** 3)
    lap = 0.1 - 0.06 + 0.02 + 0.012 * x + 0.018 * z
    for stencil in (7, 19):
        cfg = _cfg19((nx, ny, nz), D=D, dt=dt, h=h)
        cfg["stencil"] = stencil
        out = orc.run(cfg, c[None], 1)[0]
        inner = (slice(1, -1),) * 3
        np.testing.assert_allclose(out[inner], (c + dt * D * lap)[inner], rtol=0, atol=1e-14)


def test_stencil19_isotropy_beats_seven_point(orc):
    # the paper's reason for eq. (3): equal |k| in different directions decays
    # at nearly equal rates.  Wave vectors (5,0,0) and (3,4,0) on a 40^2 x 4
    # periodic grid have the same |k|; the spread of their measured decay
    # rates must be far smaller than with the 7-point stencil
    nx, ny, nz = 40, 40, 4
    D, dt = 1.0, 0.05
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    rates = {}
    for stencil in (7, 19):
        cfg = _cfg19((nx, ny, nz), D=D, dt=dt, bc="periodic")
        cfg["stencil"] = stencil
        for m in ((5, 0), (3, 4)):
            mode = np.cos(2 * np.pi * (m[0] * x + m[1] * y) / nx)
            out = orc.run(cfg, mode[None], 1)[0]
            g = float((out * mode).sum() / (mode * mode).sum())
            rates[stencil, m] = (1.0 - g) / (D * dt)
    k2 = (2 * np.pi * 5 / nx) ** 2
    for stencil in (7, 19):
        assert abs(rates[stencil, (5, 0)] - k2) < 0.06 * k2
    spread7 = abs(rates[7, (5, 0)] - rates[7, (3, 4)])
    spread19 = abs(rates[19, (5, 0)] - rates[19, (3, 4)])
    assert spread19 < spread7 / 20.0


@pytest.mark.parametrize("factor,grows", [(1.0 + 1e-2, True), (1.0 - 1e-2, False)])
def test_stencil19_stability_bound(orc, factor, grows):
    # the symbol's minimum over the cube of cosines is -32, at two cosines -1
    # and one +1: the x-y checkerboard, constant in z, has g = 1 - (16/3) r
    # (r = D dt / h^2) and stays bounded iff r <= 3/8; the full 3-D
    # checkerboard has g = 1 - 4 r
    n = 8
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    cb2 = ((-1.0) ** (x + y))[None]
    cb3 = ((-1.0) ** (x + y + z))[None]
    dt = factor * 3.0 / 8.0
    cfg = _cfg19((n, n, n), dt=dt, bc="periodic")
    out = orc.run(cfg, cb2, 150)
    np.testing.assert_allclose(out, (1.0 - 16.0 / 3.0 * dt) ** 150 * cb2, rtol=1e-10, atol=0)
    assert (np.abs(out).max() > 1.0) == grows
    out3 = orc.run(cfg, cb3, 7)
    np.testing.assert_allclose(out3, (1.0 - 4.0 * dt) ** 7 * cb3, rtol=1e-12, atol=0)


@pytest.mark.parametrize("bc", ["neumann", "periodic"])
def test_stencil19_mass_conserved(orc, bc):
    cfg = _cfg19((9, 6, 7), D=0.9, dt=0.1, bc=bc)
    c0 = W.initial_fields(W.with_(cfg, init="uniform_noise"), seed=13).astype(np.float64)
    out = orc.run(cfg, c0, 30)
    assert abs(out.sum() - c0.sum()) <= 1e-12 * abs(c0.sum())
    assert not np.allclose(out, c0)


# --------------------------------------------------------------------------
# Table 1, row 4: the plume's three-axis, time-dependent wind
# --------------------------------------------------------------------------
def _plume_cfg(shape, **kw):
    cfg = W.plume(shape=shape, src=(0, 0, 0), **kw)
    return cfg


def test_plume_linear_field_follows_uz_of_t(orc):
    # c = z h is linear in z and uniform in x, y: away from the z faces the
    # upwind difference is 1/h for either sign of u_z and the Laplacian is 0,
    # so each step subtracts dt u_z(t_k) with t_k = k dt at the step's start;
    # the run crosses a sign change of sin(t / tau)
    nx, ny, nz = 4, 5, 40
    dt, h, tau, amp = 5.0, 100.0, 20.0, 5.0
    cfg = _plume_cfg((nx, ny, nz), dt=dt, h=h, uz_tau=tau, uz_amp=amp, E=0.0)
    z = np.arange(nz) * h
    c0 = np.broadcast_to(z[:, None, None], (nz, ny, nx))[None].copy()
    n0, n = 3, 16
    out = orc.run(cfg, c0, n, n0=n0)
    drift = dt * sum(amp * math.sin(k * dt / tau) for k in range(n0, n0 + n))
    assert any(math.sin(k * dt / tau) < 0 for k in range(n0, n0 + n))
    inner = slice(n + 1, nz - n - 1)
    np.testing.assert_allclose(out[0, inner], c0[0, inner] - drift, rtol=0, atol=1e-9)


@pytest.mark.parametrize("impl", ["c", "np"])
def test_plume_mass_budget_periodic(orc, impl):
    # periodic faces: upwind advection along every axis and diffusion move
    # mass around but conserve it; the point source adds exactly E dt per step
    cfg = _plume_cfg((6, 5, 7), dt=5.0, E=10.0)
    cfg["bc"] = [["periodic"] * 6]
    cfg["source"] = dict(x=2, y=3, z=4, species=0, rate=10.0)
    c0 = W.uniform01(4, 0, 6 * 5 * 7).reshape(1, 7, 5, 6)
    run = orc.run if impl == "c" else orc.np_run
    out = run(cfg, c0, 25, 7)
    assert out.sum() == pytest.approx(c0.sum() + 25 * 10.0 * 5.0, rel=1e-13)


def _upwind_pair(n, periodic, u):
    # 1-D matrix of -u d/dx, backward difference for u > 0, forward for u < 0,
    # zero gradient beyond a zero-flux face
    if u > 0:
        B = -np.eye(n) + np.eye(n, k=-1)
        if periodic:
            B[0, -1] = 1.0
        else:
            B[0, 0] = 0.0
        return u * B
    if u < 0:
        F = np.eye(n, k=1) - np.eye(n)
        if periodic:
            F[-1, 0] = 1.0
        else:
            F[-1, -1] = 0.0
        return -u * F
    return np.zeros((n, n))


@pytest.mark.parametrize("bc", ["neumann", "periodic"])
def test_plume_dense_operator_product(orc, bc):
    # c_{k+1} = (I + dt A(t_k)) c_k + dt E e_src, with A(t) the Kronecker sum
    # of the 7-point Laplacian and the three upwind matrices of u(t)
    nx, ny, nz = 3, 4, 5
    per = bc == "periodic"
    D, h, dt, tau = 0.3, 1.0, 0.1, 0.25
    ux, uy, amp = 0.7, -0.4, 0.9
    cfg = _plume_cfg((nx, ny, nz), D=D, h=h, dt=dt, ux=ux, uy=uy, uz_amp=amp, uz_tau=tau,
                     E=2.0)
    cfg["bc"] = [[bc] * 6]
    cfg["source"] = dict(x=1, y=2, z=3, species=0, rate=2.0)
    Ix, Iy, Iz = np.eye(nx), np.eye(ny), np.eye(nz)
    L = (np.kron(Iz, np.kron(Iy, _lap1d(nx, per))) + np.kron(Iz, np.kron(_lap1d(ny, per), Ix))
         + np.kron(_lap1d(nz, per), np.kron(Iy, Ix))) / h ** 2
    e = np.zeros(nx * ny * nz)
    e[(3 * ny + 2) * nx + 1] = 1.0
    c = W.uniform01(8, 0, nx * ny * nz)
    c0 = c.copy()
    n = 12
    for k in range(n):
        uz = amp * math.sin(k * dt / tau)
        A = (D * L + np.kron(Iz, np.kron(Iy, _upwind_pair(nx, per, ux))) / h
             + np.kron(Iz, np.kron(_upwind_pair(ny, per, uy), Ix)) / h
             + np.kron(_upwind_pair(nz, per, uz), np.kron(Iy, Ix)) / h)
        c = c + dt * (A @ c) + dt * 2.0 * e
    out = orc.run(cfg, c0.reshape(1, nz, ny, nx), n).ravel()
    np.testing.assert_allclose(out, c, rtol=0, atol=1e-12)


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_plume_courant_one_shifts_along_y(orc, sign):
    # u_y = +-h/dt, no diffusion, no u_x or u_z: an exact shift of one cell
    # per step along y, in the direction of the wind
    cfg = _plume_cfg((4, 9, 3), D=0.0, dt=2.0, h=1.0, ux=0.0, uy=sign * 0.5, uz_amp=0.0,
                     E=0.0)
    cfg["bc"] = [["periodic"] * 6]
    c0 = W.uniform01(2, 0, 4 * 9 * 3).reshape(1, 3, 9, 4)
    out = orc.run(cfg, c0, 5)
    np.testing.assert_array_equal(out, np.roll(c0, int(sign) * 5, axis=2))


# --------------------------------------------------------------------------
# Table 1, row 3: Cahn-Hilliard with lambda, eps, gamma, sigma and a sink
# --------------------------------------------------------------------------
def _lam_of(theta, stencil, h):
    if stencil == 7:
        return sum(4.0 * math.sin(t / 2) ** 2 for t in theta) / h ** 2
    return -_symbol19(theta) / (6.0 * h ** 2)


@pytest.mark.parametrize("stencil", [7, 19])
def test_ch_table1_linear_symbol(orc, stencil):
    # no reaction (c1 = c2 = 0); about cbar the mode's amplitude follows
    # g = 1 + dt lambda L (eps - 3 gamma cbar^2 - sigma L), L the stencil's
    # symbol: c3' = -lambda Lap(eps c - gamma c^3 + sigma Lap c) linearised
    n = 12
    cbar, dt = 0.3, 0.01
    cfg = W.ch_table1(shape=(n, n, 4), stencil=stencil, dt=dt, lam=0.8, eps=1.3, gamma=0.9,
                      sigma=0.6)
    cfg["bc"] = [["periodic"] * 6 for _ in range(3)]
    P = cfg["params"]
    z, y, x = np.meshgrid(np.arange(4), np.arange(n), np.arange(n), indexing="ij")
    th = (2 * np.pi * 3 / n, 2 * np.pi * 1 / n, 0.0)
    mode = np.cos(th[0] * x + th[1] * y)
    amp = 1e-8
    c0 = np.stack([np.zeros_like(mode), np.zeros_like(mode), cbar + amp * mode])
    steps = 30
    out = orc.run(cfg, c0, steps)
    L = _lam_of(th, stencil, cfg["h"])
    g = 1.0 + dt * P["lam"] * L * (P["eps"] - 3.0 * P["gamma"] * cbar ** 2 - P["sigma"] * L)
    # the uniform part follows the scalar map of -lambda Lap(...) = 0: it stays cbar
    np.testing.assert_allclose(out[2] - cbar, amp * g ** steps * mode, rtol=0, atol=1e-15)


@pytest.mark.parametrize("stencil,grows", [(7, True), (19, False)])
def test_ch_table1_time_step_needs_the_19_point_stencil(orc, stencil, grows):
    # Table 1's dt = 0.02 (h = 1, lambda = eps = gamma = sigma = 1) about
    # c = 0: the fastest mode of each stencil (7-point: the 3-D checkerboard,
    # L = 12; 19-point: the x-y checkerboard, L = 16/3) has
    # g = 1 + dt L (1 - L): -1.64 (grows) and 0.54 (decays)
    n = 8
    cfg = W.ch_table1(shape=(n, n, n), stencil=stencil, k1=0.0, k2=0.0)
    cfg["bc"] = [["periodic"] * 6 for _ in range(3)]
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    mode = (-1.0) ** (x + y + z) if stencil == 7 else (-1.0) ** (x + y)
    L = 12.0 if stencil == 7 else 16.0 / 3.0
    amp = 1e-9
    c0 = np.stack([np.zeros_like(mode), np.zeros_like(mode), amp * mode])
    steps = 20
    out = orc.run(cfg, c0, steps)
    g = 1.0 + cfg["dt"] * L * (1.0 - L)
    np.testing.assert_allclose(out[2], amp * g ** steps * mode, rtol=1e-9, atol=0)
    assert (abs(g) > 1.0) == grows


def test_ch_table1_budgets(orc):
    # zero flux everywhere: with k1 = k2 = 0, sum c3 is conserved; with
    # k2 = 0 and D1 = D2, sum (c1 - c2) and sum (c2 + c3) are conserved
    cfg = W.ch_table1(shape=(9, 7, 6), stencil=19, dt=0.01)
    cfg["bc"] = [["neumann"] * 6 for _ in range(3)]
    c0 = W.initial_fields(W.with_(cfg, init="uniform_noise"), seed=21).astype(np.float64)
    c0[2] = 2.0 * c0[2] - 1.0
    a = orc.run(W.with_(cfg, params=dict(cfg["params"], k1=0.0, k2=0.0)), c0, 25)
    assert a[2].sum() == pytest.approx(c0[2].sum(), rel=1e-12, abs=1e-12)
    assert not np.allclose(a[2], c0[2])
    b = orc.run(W.with_(cfg, params=dict(cfg["params"], k2=0.0)), c0, 25)
    assert (b[0] - b[1]).sum() == pytest.approx((c0[0] - c0[1]).sum(), rel=1e-12, abs=1e-12)
    assert (b[1] + b[2]).sum() == pytest.approx((c0[1] + c0[2]).sum(), rel=1e-12, abs=1e-12)
    assert (b[1].sum() - c0[1].sum()) < -1e-3                     # the reaction ran


def test_oracles_agree_on_every_family(orc):
    cases = [W.diffusion_blob(8), W.brusselator(8), W.ch_front(8),
             W.air((8, 8, 8), src=(3, 4, 2)),
             W.brusselator(shape=(7, 9, 6), bc="neumann"),
             W.ch_front(shape=(9, 7, 10)), W.air((11, 6, 5), src=(10, 0, 4)),
             W.with_(W.brusselator(shape=(7, 9, 6), bc="neumann"), stencil=19),
             W.with_(W.brusselator(8), stencil=19),
             W.with_(W.air((9, 7, 6), src=(8, 1, 3)), stencil=19, D=[[0.1] * 3] * 3),
             W.with_(W.ch_front(shape=(8, 7, 9)), stencil=19),
             W.turing(shape=(9, 8, 7)), W.turing(shape=(7, 9, 8), stencil=19),
             W.plume(shape=(9, 8, 10), src=(2, 3, 4)),
             W.with_(W.plume(shape=(8, 9, 7), src=(5, 1, 2)), stencil=19),
             W.ch_table1(shape=(9, 8, 7), dt=0.005), W.ch_table1(shape=(8, 7, 9), stencil=7,
                                                                 dt=0.005)]
    for cfg in cases:
        f = W.initial_fields(cfg)
        a = orc.run(cfg, f, 9)
        b = orc.np_run(cfg, f, 9)
        np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12 * np.abs(a).max())
