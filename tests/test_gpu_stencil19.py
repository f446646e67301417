"""The 19-point Laplacian of eqs. (3)-(4) on the GPU against the FP64 oracle,
through the C ABI.

Tolerances as in ``test_gpu_parity``: normwise max relative error 1e-5 for
pure diffusion and 1e-4 for the nonlinear problems (FP32 state).  Every
case first checks that the oracle's 19-point and 7-point results differ by
far more than the tolerance, so the comparison can tell the stencils apart.
Tilings and z-chunks evaluate the same per-cell arithmetic on the same
inputs, so they must agree bit for bit.
"""
import numpy as np
import pytest

from paper_1004_0480_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_DIFF = 1e-5
TOL_NONLIN = 1e-4
SHAPE = (141, 23, 19)   # 3 x tiles of 64 (ragged 13), ragged y tiles and z chunks


@pytest.fixture(scope="module")
def rd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1004_0480_gb300 import build as B
    B.build()
    from paper_1004_0480_gb300 import sim
    return sim


def rel_err(got, ref):
    return max(float(np.abs(got[s] - ref[s]).max() / max(np.abs(ref[s]).max(), 1e-30))
               for s in range(ref.shape[0]))


def run_gpu(rd, cfg, steps, storage="f32", tuning=None, fields=None):
    f = W.initial_fields(cfg) if fields is None else fields
    with rd.Sim(cfg, storage) as sim:
        if tuning:
            sim.set_tuning(**tuning)
        sim.set_fields(f)
        sim.step(steps)
        return sim.get_fields()


def s19(cfg, **kw):
    return W.with_(cfg, stencil=19, **kw)


def family_cases():
    per_d = s19(W.diffusion_blob(shape=SHAPE))
    per_d["bc"] = [["periodic"] * 6]
    noise_d = s19(W.diffusion_blob(shape=(70, 37, 23), dt=0.2), init="uniform_noise")
    mixed_b = s19(W.brusselator(shape=SHAPE))
    mixed_b["bc"] = [["periodic", "periodic", "neumann", "neumann", "neumann", "neumann"]] * 2
    air_iso = s19(W.air(SHAPE, src=(5, 17, 2)), D=[[0.1] * 3] * 3)
    air_held = s19(W.air(SHAPE, src=(100, 3, 11)), D=[[0.12] * 3] * 3)
    air_held["bc"] = [["neumann", "neumann", "periodic", "periodic", "neumann", "dirichlet"]] * 3
    air_held["bc_value"] = [[0.0] * 5 + [v] for v in (0.0, 0.02, 1.0)]
    air_held["wind"] = dict(kind="const", u0=-0.5)
    # nx % 4 == 3: the last vector of a row holds three cells, so the +x
    # diagonals of its cells come from clamped neighbour-row elements; ny a
    # multiple of the 4- and 6-row tiles puts the last tile's halo row on
    # the y ghost row
    neu67 = s19(W.brusselator(shape=(67, 24, 19), bc="neumann"))
    mixed67 = s19(W.air((67, 24, 19), src=(66, 23, 5)), D=[[0.1] * 3] * 3)
    mixed67["bc"] = [["neumann", "neumann", "neumann", "neumann", "periodic", "periodic"]] * 3
    mixed67["wind"] = dict(kind="const", u0=0.4)
    return {
        "brusselator_neumann_nx67": (neu67, TOL_NONLIN),
        "air_mixed_bc_nx67": (mixed67, TOL_NONLIN),
        "diffusion_neumann": (s19(W.diffusion_blob(shape=SHAPE)), TOL_DIFF),
        "diffusion_periodic": (per_d, TOL_DIFF),
        "diffusion_noise_neumann": (noise_d, TOL_DIFF),
        "brusselator_periodic": (s19(W.brusselator(shape=SHAPE)), TOL_NONLIN),
        "brusselator_neumann": (s19(W.brusselator(shape=SHAPE, bc="neumann")), TOL_NONLIN),
        "brusselator_mixed_bc": (mixed_b, TOL_NONLIN),
        "air_wind_source": (air_iso, TOL_NONLIN),
        "air_held_top_reverse_wind": (air_held, TOL_NONLIN),
        # Table 1 parameters with larger initial noise (the paper's +-5e-4
        # would not separate the stencils in 13 steps)
        "turing_table1": (W.turing(shape=SHAPE, stencil=19, sigma=0.3), TOL_NONLIN),
    }


CASES = family_cases()
TILINGS = [
    dict(tsteps=1, tile_q=16, tile_y=4, zchunk=5, graph=0),
    dict(tsteps=1, tile_q=16, tile_y=6, zchunk=19, graph=1),
    dict(tsteps=1, tile_q=16, tile_y=14, zchunk=7, graph=1),
    dict(tsteps=1, tile_q=16, tile_y=16, zchunk=8, graph=0),
    dict(tsteps=1, tile_q=16, tile_y=30, zchunk=3, graph=1),
]


@pytest.mark.parametrize("name", sorted(CASES))
def test_stencil19_matches_oracle_and_tilings_agree_bitwise(rd, orc, name):
    cfg, tol = CASES[name]
    steps = 13
    f = W.initial_fields(cfg)
    ref = orc.run(cfg, f, steps)
    ref7 = orc.run(W.with_(cfg, stencil=7), f, steps)
    assert rel_err(ref7, ref) > 10 * tol, "case does not separate the stencils"
    outs = []
    for t in TILINGS:
        got = run_gpu(rd, cfg, steps, tuning=t, fields=f)
        err = rel_err(got, ref)
        assert err <= tol, f"{name} {t}: rel err {err:.3e}"
        outs.append(got)
    for o in outs[1:]:
        assert np.array_equal(o.view(np.uint32), outs[0].view(np.uint32)), \
            f"{name}: tilings disagree bitwise"


@pytest.mark.parametrize("name", ["diffusion_neumann", "brusselator_periodic",
                                  "air_wind_source"])
def test_stencil19_bf16_storage(rd, orc, name):
    cfg, _ = CASES[name]
    steps = 10
    f = W.initial_fields(cfg)
    ref = orc.run(cfg, f, steps)
    outs = [run_gpu(rd, cfg, steps, storage="bf16", tuning=t, fields=f) for t in TILINGS[:3]]
    for o in outs[1:]:
        assert np.array_equal(o.view(np.uint32), outs[0].view(np.uint32))
    # bf16 keeps 8 bits of mantissa: a few ulps of 2^-8 after 10 steps
    assert rel_err(outs[0], ref) < 3e-2


def test_stencil19_periodic_x_not_a_multiple_of_four(rd, orc):
    # nx = 66: the last x tile holds half a vector of real cells and its
    # right halo (and the corner vectors) wrap to x = 0 element by element
    cfg = s19(W.brusselator(shape=(66, 20, 9)))
    f = W.initial_fields(cfg)
    ref = orc.run(cfg, f, 9)
    got = run_gpu(rd, cfg, 9, tuning=dict(tile_y=6, zchunk=4, graph=0), fields=f)
    assert rel_err(got, ref) <= TOL_NONLIN


@pytest.mark.parametrize("bc", ["neumann", "periodic"])
def test_stencil19_smallest_grid(rd, orc, bc):
    cfg = s19(W.brusselator(shape=(2, 2, 2), bc=bc))
    f = W.initial_fields(cfg)
    assert rel_err(run_gpu(rd, cfg, 5, fields=f), orc.run(cfg, f, 5)) <= TOL_NONLIN


def test_stencil19_brusselator_200_steps(rd, orc):
    cfg = s19(W.brusselator(shape=(96, 40, 24)))
    f = W.initial_fields(cfg)
    ref = orc.run(cfg, f, 200)
    for t in (None, dict(tile_y=8, zchunk=6, graph=1)):
        assert rel_err(run_gpu(rd, cfg, 200, tuning=t, fields=f), ref) <= TOL_NONLIN


def test_stencil19_tuning_rules(rd):
    from paper_1004_0480_gb300 import _lib as L
    cfg = s19(W.brusselator(shape=(64, 16, 8)))
    with rd.Sim(cfg) as sim:
        assert sim.tuning()["tsteps"] == 1
        with pytest.raises(Exception):
            sim.set_tuning(tsteps=2)          # one step per launch
        with pytest.raises(Exception):
            sim.set_tuning(tile_y=5)          # whole halo warp: even heights
        with pytest.raises(Exception):
            sim.set_tuning(tile_y=32)         # at most 512 threads
        # a batch takes 19-point members (of one stencil: a 7-point context
        # cannot join them)
        b = rd.Batch("brusselator")
        other = rd.Sim(W.brusselator(shape=(64, 16, 8)))
        try:
            assert sim.lib.rd_batch_add(b.b, sim.ctx) == L.RD_OK
            assert sim.lib.rd_batch_add(b.b, other.ctx) == L.RD_EINVAL
        finally:
            b.close()
            other.close()


def test_stencil19_autotune_and_full_size_step(rd, orc):
    # the 256^3 Brusselator with the paper's stencil, autotuned, one step
    # against the oracle on the whole grid
    cfg = s19(W.cfg_brusselator_256())
    f = W.initial_fields(cfg)
    ref = orc.run(cfg, f, 1)
    with rd.Sim(cfg) as sim:
        t = sim.autotune()
        assert t["tsteps"] == 1 and t["tile_y"] % 2 == 0
        sim.set_fields(f)
        sim.step(1)
        got = sim.get_fields()
    assert rel_err(got, ref) <= TOL_NONLIN
