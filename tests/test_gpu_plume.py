"""The inert plume of Table 1, row 4, on the GPU against the FP64 oracle:
first-order upwind along all three axes with u = (5, 1, 5 sin(t / 500))
m/s, t = n dt at the start of step n, D = 100 m^2/s, h = 100 m, dt = 5 s,
a point emission of 10 per second, zero flux, with both stencils.

u_z changes sign at t = 500 pi s (step 314.16), so the runs start at step
250 (rd_set_step_count) and cross it.  The step index lives on the device
per context and time level, so graph replay, calls of any length, and
batches whose members are at different times must all give the same bits.
Tolerance: normwise 1e-4 (the problem is linear; FP32 state).
"""
import numpy as np
import pytest

from paper_1004_0480_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-4
N0 = 250


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


def plume(shape=(70, 36, 40), stencil=7, noise=True, src=(20, 18, 9)):
    cfg = W.plume(shape=shape, src=src)
    cfg["stencil"] = stencil
    if noise:
        cfg["init"] = "uniform_noise"
    return cfg


def run_gpu(rd, cfg, steps, n0=N0, tuning=None, fields=None, chunks=None):
    f = W.initial_fields(cfg) if fields is None else fields
    with rd.Sim(cfg) as sim:
        if tuning:
            sim.set_tuning(**tuning)
        sim.lib.rd_set_step_count(sim.ctx, n0)
        sim.set_fields(f)
        for n in (chunks or [steps]):
            sim.step(n)
        assert sim.steps_done == n0 + steps
        return sim.get_fields()


TILINGS = [
    dict(tsteps=1, tile_q=16, tile_y=4, zchunk=5, graph=0),
    dict(tsteps=1, tile_q=16, tile_y=6, zchunk=40, graph=1),
    dict(tsteps=1, tile_q=16, tile_y=14, zchunk=7, graph=1),
]


@pytest.mark.parametrize("stencil", [7, 19])
def test_plume_across_the_sign_change_of_uz(rd, orc, stencil):
    cfg = plume(stencil=stencil)
    steps = 130                       # steps 250 .. 379: u_z < 0 from step 315
    f = W.initial_fields(cfg)
    ref = orc.run(cfg, f, steps, n0=N0)
    # the same run with u_z switched off must differ: the comparison sees
    # the vertical wind
    frozen = W.with_(cfg, wind=dict(cfg["wind"], uz_tau=1e12))
    assert rel_err(orc.run(frozen, f, steps, n0=N0), ref) > 100 * TOL
    outs = []
    for t in TILINGS:
        got = run_gpu(rd, cfg, steps, tuning=t, fields=f)
        err = rel_err(got, ref)
        assert err <= TOL, f"{t}: rel err {err:.3e}"
        outs.append(got)
    for o in outs[1:]:
        assert np.array_equal(o.view(np.uint32), outs[0].view(np.uint32))
    # calls of any length (graph replays and plain launches mixed)
    split = run_gpu(rd, cfg, steps, tuning=TILINGS[1], fields=f, chunks=[1, 37, 16, 3, 73])
    assert np.array_equal(split.view(np.uint32), outs[0].view(np.uint32))


def test_plume_from_rest_with_the_paper_source(rd, orc):
    # the paper's start: c = 0, the emission at one cell; 200 steps from t = 0
    cfg = plume(shape=(64, 48, 96), noise=False, src=(16, 24, 12), stencil=19)
    f = W.initial_fields(cfg)
    ref = orc.run(cfg, f, 200)
    got = run_gpu(rd, cfg, 200, n0=0, fields=f)
    assert rel_err(got, ref) <= TOL
    assert got.min() >= 0.0


def test_plume_batch_members_at_different_times(rd):
    cfgs = [plume(shape=(70, 36, 40)), plume(shape=(33, 50, 21), src=(3, 40, 5)),
            plume(shape=(64, 20, 30), src=(60, 1, 28))]
    n0s = [N0, 0, 301]
    steps = 37
    tun = dict(tsteps=1, tile_q=16, tile_y=6, zchunk=8, graph=1)
    ref = [run_gpu(rd, c, steps, n0=n, tuning=tun) for c, n in zip(cfgs, n0s)]
    sims = [rd.Sim(c) for c in cfgs]
    try:
        for c, s, n in zip(cfgs, sims, n0s):
            s.lib.rd_set_step_count(s.ctx, n)
            s.set_fields(W.initial_fields(c))
        b = rd.Batch("diffusion")
        b.set_tuning(**tun)
        for s in sims:
            b.add(s)
        b.step(20)
        b.step(17)
        b.sync()
        for s, r, n in zip(sims, ref, n0s):
            assert s.steps_done == n + steps
            assert np.array_equal(s.get_fields(), r)
        b.close()
    finally:
        for s in sims:
            s.close()


def test_plume_full_grid_few_steps(rd, orc):
    # the paper's 144 x 144 x 384 grid, 19-point stencil, three steps
    cfg = plume(shape=(144, 144, 384), stencil=19, src=None)
    f = W.initial_fields(cfg)
    ref = orc.run(cfg, f, 3, n0=N0)
    with rd.Sim(cfg) as sim:
        sim.autotune()
        sim.lib.rd_set_step_count(sim.ctx, N0)
        sim.set_fields(f)
        sim.step(3)
        got = sim.get_fields()
    assert rel_err(got, ref) <= TOL


def test_plume_refusals(rd):
    from paper_1004_0480_gb300 import _lib as L
    cfg = plume()
    with rd.Sim(cfg) as sim:
        with pytest.raises(L.RdError):
            sim.set_tuning(tsteps=2)          # one step per launch
    bad = W.with_(cfg, wind=dict(cfg["wind"], uz_tau=0.0))
    with pytest.raises(L.RdError) as e:
        rd.Sim(bad)
    assert e.value.status == L.RD_EINVAL
    fast = W.with_(cfg, wind=dict(cfg["wind"], ux=50.0))   # Courant 2.5 along x
    with pytest.raises(L.RdError) as e:
        rd.Sim(fast)
    assert e.value.status == L.RD_EUNSTABLE
