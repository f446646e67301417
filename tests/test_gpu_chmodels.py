"""Cahn-Hilliard models and batches on the 19-point stencil, through the C
ABI, against the FP64 oracle.

  * The phase separation behind a front of Table 1, row 3 (c1 + c2 -> c3,
    the sink k2 c1 c3, c3 moved by -lambda Lap(eps c3 - gamma c3^3 +
    sigma Lap c3), c1 held at 10 on the x = 0 layer) on the 7-point kernels
    (one and two steps per launch) and on the 19-point stencil.
  * The front model on the 19-point stencil (eqs. (3)-(4)): two launches
    per step, mu and then the update (Section 4.1, "Laplacian, boundary
    rule, Laplacian").
  * Batches of 19-point contexts: bit for bit the standalone result.
  * The paper's own time step for row 3 (dt = 0.02, h = 1) is within the
    explicit bound only with the 19-point stencil: rejected on the 7-point
    one, 200 steps within 1e-4 of the oracle on the 19-point one.

Tolerances as in test_gpu_parity: normwise 1e-4 for the nonlinear problems
(FP32 state, <= 200 steps); tilings and batches must agree bit for bit.
"""
import numpy as np
import pytest

from paper_1004_0480_gb300 import workloads as W

pytestmark = pytest.mark.gpu

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


def table1(shape=SHAPE, dt=0.01, stencil=7, noise=True, **kw):
    """Table 1 row 3 with its parameters; dt 0.01 is within the 7-point
    bound (dt lambda L (sigma L + 2) = 1.68 <= 2 with L = 12); ``noise``
    starts every species from U[0,1) (so the Cahn-Hilliard term acts from
    the first step), else from the paper's c1 = 0, c2 = 1, c3 = -1."""
    cfg = W.ch_table1(shape=shape, dt=dt, stencil=stencil, **kw)
    if noise:
        cfg["init"] = "uniform_noise"
    return cfg


TILINGS7 = [
    dict(tsteps=1, tile_q=16, tile_y=4, zchunk=5, graph=0),
    dict(tsteps=2, tile_q=16, tile_y=5, zchunk=7, graph=0),
    dict(tsteps=2, tile_q=16, tile_y=8, zchunk=19, graph=1),
    dict(tsteps=1, tile_q=16, tile_y=12, zchunk=8, graph=1),
]
TILINGS19 = [
    dict(tsteps=1, tile_q=16, tile_y=4, zchunk=5, graph=0),
    dict(tsteps=1, tile_q=16, tile_y=6, zchunk=19, graph=1),
    dict(tsteps=1, tile_q=16, tile_y=12, zchunk=7, graph=1),
    dict(tsteps=1, tile_q=16, tile_y=16, zchunk=8, graph=0),
]


def cases19():
    front = W.with_(W.ch_front(shape=SHAPE), stencil=19)
    front_per = W.with_(front, init="uniform_noise",
                        bc=[["periodic"] * 6 for _ in range(3)],
                        bc_value=[[0.0] * 6 for _ in range(3)])
    front_src = W.with_(front, source={"x": 70, "y": 11, "z": 9, "species": 1, "rate": 2.0})
    mixed = table1(stencil=19)
    mixed["bc"] = [["neumann", "neumann", "periodic", "periodic", "neumann", "neumann"]] * 3
    mixed["bc_value"] = [[0.0] * 6 for _ in range(3)]
    return {
        "front_19": front,
        "front_19_periodic": front_per,
        "front_19_source_on_b": front_src,
        "table1_19": table1(stencil=19),
        "table1_19_periodic_y": mixed,
    }


CASES19 = cases19()


def test_table1_model_7pt_tilings_and_depths(rd, orc):
    cfg = table1()
    steps = 13
    f = W.initial_fields(cfg)
    ref = orc.run(cfg, f, steps)
    outs = []
    for t in TILINGS7:
        got = run_gpu(rd, cfg, steps, tuning=t, fields=f)
        err = rel_err(got, ref)
        assert err <= TOL_NONLIN, f"{t}: rel err {err:.3e}"
        outs.append(got)
    for o in outs[1:]:
        assert np.array_equal(o.view(np.uint32), outs[0].view(np.uint32))


def test_table1_model_7pt_paper_start_200_steps(rd, orc):
    # the paper's initial state (c3 = -1 everywhere: mu = 0 away from the
    # front) and its held layer c1 = 10 at x = 0
    cfg = table1(shape=(70, 24, 20), noise=False)
    f = W.initial_fields(cfg)
    ref = orc.run(cfg, f, 200)
    got = run_gpu(rd, cfg, 200, fields=f)
    assert rel_err(got, ref) <= TOL_NONLIN
    assert np.all(got[0][:, :, 0] == 10.0)


@pytest.mark.parametrize("name", sorted(CASES19))
def test_ch_19pt_matches_oracle_and_tilings_agree_bitwise(rd, orc, name):
    cfg = CASES19[name]
    steps = 13
    f = W.initial_fields(cfg)
    ref = orc.run(cfg, f, steps)
    ref7 = orc.run(W.with_(cfg, stencil=7), f, steps)
    assert rel_err(ref7, ref) > 10 * TOL_NONLIN, "case does not separate the stencils"
    outs = []
    for t in TILINGS19:
        got = run_gpu(rd, cfg, steps, tuning=t, fields=f)
        err = rel_err(got, ref)
        assert err <= TOL_NONLIN, f"{name} {t}: rel err {err:.3e}"
        outs.append(got)
    for o in outs[1:]:
        assert np.array_equal(o.view(np.uint32), outs[0].view(np.uint32)), \
            f"{name}: tilings disagree bitwise"


@pytest.mark.parametrize("name", ["front_19", "table1_19"])
def test_ch_19pt_bf16_storage(rd, orc, name):
    cfg = CASES19[name]
    f = W.initial_fields(cfg)
    ref = orc.run(cfg, f, 10)
    outs = [run_gpu(rd, cfg, 10, storage="bf16", tuning=t, fields=f) for t in TILINGS19[:2]]
    assert np.array_equal(outs[0].view(np.uint32), outs[1].view(np.uint32))
    assert rel_err(outs[0], ref) < 3e-2


def test_ch_19pt_two_launches_per_step(rd):
    cfg = CASES19["front_19"]
    with rd.Sim(cfg, tuning=dict(graph=0)) as sim:
        sim.set_fields(W.initial_fields(cfg))
        l0 = sim.launches
        sim.step(5)
        assert sim.launches - l0 == 10


def test_table1_paper_dt_needs_the_19_point_stencil(rd, orc):
    from paper_1004_0480_gb300 import _lib as L
    with pytest.raises(L.RdError) as e:
        rd.Sim(W.ch_table1(shape=(16, 16, 16), stencil=7))
    assert e.value.status == L.RD_EUNSTABLE
    # the paper's dt = 0.02 with its 19-point stencil: 200 steps from the
    # paper's initial state and from noise
    for noise in (False, True):
        cfg = table1(shape=(48, 40, 36), dt=0.02, stencil=19, noise=noise)
        f = W.initial_fields(cfg)
        ref = orc.run(cfg, f, 200)
        got = run_gpu(rd, cfg, 200, fields=f)
        assert rel_err(got, ref) <= TOL_NONLIN, f"noise={noise}"


def test_front_19pt_200_steps(rd, orc):
    cfg = W.with_(W.ch_front(48), stencil=19)
    f = W.initial_fields(cfg)
    ref = orc.run(cfg, f, 200)
    assert rel_err(run_gpu(rd, cfg, 200, fields=f), ref) <= TOL_NONLIN


BATCH_SIZES = [(23, 17, 11), (140, 9, 14), (16, 33, 25), (70, 20, 8)]


def batch_cfgs(model):
    mk = {"diffusion": lambda s, i: W.diffusion_blob(shape=s, seed=i),
          "brusselator": lambda s, i: W.brusselator(shape=s, seed=i),
          "air": lambda s, i: W.with_(W.air(s, src=(1, 2, 3), seed=i), D=[[0.1] * 3] * 3),
          "turing": lambda s, i: W.turing(shape=s, seed=i, sigma=0.3),
          "ch_front": lambda s, i: W.ch_front(shape=s, seed=i),
          "ch_table1": lambda s, i: table1(shape=s, seed=i)}[model]
    return [W.with_(mk(s, i), stencil=19) for i, s in enumerate(BATCH_SIZES)]


@pytest.mark.parametrize("model", ["diffusion", "brusselator", "air", "turing", "ch_front",
                                   "ch_table1"])
def test_batch_19pt_matches_standalone_bitwise(rd, orc, model):
    cfgs = batch_cfgs(model)
    steps = 21            # one 16-launch graph replay and 5 plain launches
    tun = dict(tsteps=1, tile_q=16, tile_y=4, zchunk=6, graph=1)
    ref = [run_gpu(rd, c, steps, tuning=tun) for c in cfgs]
    sims = [rd.Sim(c) for c in cfgs]
    try:
        for c, s in zip(cfgs, sims):
            s.set_fields(W.initial_fields(c))
        b = rd.Batch(model)
        b.set_tuning(**tun)
        for s in sims:
            b.add(s)
        b.step(4)
        b.step(17)
        b.sync()
        for s, r in zip(sims, ref):
            assert np.array_equal(s.get_fields(), r)
        b.close()
    finally:
        for s in sims:
            s.close()
    f = W.initial_fields(cfgs[1])
    assert rel_err(ref[1], orc.run(cfgs[1], f, steps)) <= TOL_NONLIN


def test_batch_refuses_mixed_stencils(rd):
    from paper_1004_0480_gb300 import _lib as L
    a = rd.Sim(W.brusselator(shape=(16, 16, 16)))
    b = rd.Sim(W.with_(W.brusselator(shape=(16, 16, 16)), stencil=19))
    bt = rd.Batch("brusselator")
    try:
        bt.add(a)
        with pytest.raises(L.RdError) as e:
            bt.add(b)
        assert e.value.status == L.RD_EINVAL
    finally:
        bt.close()
        a.close()
        b.close()
