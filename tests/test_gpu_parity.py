"""CUDA path vs the FP64 oracle, through the C ABI.

Tolerances (normwise max relative error per species, max|g - r| / max|r|):
  pure diffusion, FP32 state      1e-5
  nonlinear problems, FP32 state  1e-4 (compared at <= 200 steps)
Different tilings, temporal-blocking depths, graph replay and batched
launches evaluate the same per-cell update on the same inputs, so they must
agree bit for bit.
"""
import numpy as np
import pytest

from paper_1004_0480_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_DIFF = 1e-5
TOL_NONLIN = 1e-4


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


SHAPE = (141, 23, 19)   # 3 x tiles of 64 (ragged 13), ragged y tiles and z chunks


def family_cases():
    neu_b = W.brusselator(shape=SHAPE, bc="neumann")
    per_d = W.diffusion_blob(shape=SHAPE)
    per_d["bc"] = [["periodic"] * 6]
    per_ch = W.ch_front(shape=SHAPE)
    per_ch["bc"] = [["periodic"] * 6 for _ in range(3)]
    per_ch["bc_value"] = [[0.0] * 6 for _ in range(3)]
    per_ch["init"] = "uniform_noise"
    per_air = W.air(SHAPE, src=(40, 0, 17))
    per_air["bc"] = [["periodic"] * 6 for _ in range(3)]
    ch_src = W.ch_front(shape=SHAPE)
    ch_src["D"][0] = [1.0, 0.5, 0.25]
    ch_src["source"] = {"x": 70, "y": 11, "z": 9, "species": 0, "rate": 2.0}
    aniso = W.diffusion_blob(shape=SHAPE)
    aniso["D"] = [[0.9, 0.3, 0.05]]
    aniso["dt"] = 0.4
    return {
        "diffusion_neumann": (W.diffusion_blob(shape=SHAPE), TOL_DIFF),
        "diffusion_periodic": (per_d, TOL_DIFF),
        "diffusion_anisotropic": (aniso, TOL_DIFF),
        "brusselator_periodic": (W.brusselator(shape=SHAPE), TOL_NONLIN),
        "brusselator_neumann": (neu_b, TOL_NONLIN),
        "ch_front_dirichlet": (W.ch_front(shape=SHAPE), TOL_NONLIN),
        "ch_periodic": (per_ch, TOL_NONLIN),
        "ch_front_aniso_source": (ch_src, TOL_NONLIN),
        "air_neumann": (W.air(SHAPE, src=(5, 17, 2)), TOL_NONLIN),
        "air_periodic": (per_air, TOL_NONLIN),
        "turing_table1": (W.turing(shape=SHAPE), TOL_NONLIN),
    }


CASES = family_cases()
TILINGS = [
    dict(tsteps=1, tile_q=16, tile_y=4, zchunk=5, graph=0),
    dict(tsteps=2, tile_q=16, tile_y=5, zchunk=7, graph=0),
    dict(tsteps=3, tile_q=16, tile_y=3, zchunk=4, graph=1),
    dict(tsteps=2, tile_q=16, tile_y=8, zchunk=19, graph=1),
    dict(tsteps=1, tile_q=16, tile_y=16, zchunk=8, graph=1),
    # 64-register one-step kernel, tile heights with compile-time variants;
    # z-chunks of 7 and 6 planes end inside and at the end of the unrolled
    # 6-plane groups
    dict(tsteps=1, tile_q=16, tile_y=8, zchunk=7, graph=1, regcap=1),
    dict(tsteps=1, tile_q=16, tile_y=16, zchunk=6, graph=0, regcap=1),
]


def tilings_for(cfg):
    if cfg["model"] == "ch_front":
        return [t for t in TILINGS if t["tsteps"] <= 2]
    return TILINGS


@pytest.mark.parametrize("name", sorted(CASES))
def test_family_matches_oracle_and_tilings_agree_bitwise(rd, orc, name):
    cfg, tol = CASES[name]
    steps = 13
    f = W.initial_fields(cfg)
    ref = orc.run(cfg, f, steps)
    outs = []
    for t in tilings_for(cfg):
        got = run_gpu(rd, cfg, steps, tuning=t, fields=f)
        err = rel_err(got, ref)
        assert err <= tol, f"{name} {t}: rel err {err:.3e}"
        outs.append(got)
    for o in outs[1:]:
        assert np.array_equal(o.view(np.uint32), outs[0].view(np.uint32)), \
            f"{name}: tilings / temporal depths disagree bitwise"


@pytest.mark.parametrize("name", ["diffusion_neumann", "brusselator_periodic",
                                  "ch_front_dirichlet", "air_neumann"])
def test_bf16_storage_is_close_and_depth_invariant(rd, orc, name):
    cfg, _ = CASES[name]
    steps = 10
    f = W.initial_fields(cfg)
    ref = orc.run(cfg, f, steps)
    outs = [run_gpu(rd, cfg, steps, storage="bf16", tuning=t, fields=f)
            for t in tilings_for(cfg)[:3]]
    for o in outs[1:]:
        assert np.array_equal(o.view(np.uint32), outs[0].view(np.uint32))
    # bf16 keeps 8 bits of mantissa: a few ulps of 2^-8 after 10 steps
    assert rel_err(outs[0], ref) < 3e-2


def test_periodic_tiles_wrapping_and_ragged(rd, orc):
    # periodic nx = 132: the x-tile at 0 wraps its left halo vector, the tile
    # at 64 has both halo vectors inside the row, the tile at 128 is ragged
    # (one vector of real cells, its right halo wraps to x = 0)
    cfg = W.brusselator(shape=(132, 20, 17))
    f = W.initial_fields(cfg)
    ref = orc.run(cfg, f, 9)
    one = run_gpu(rd, cfg, 9, tuning=dict(tsteps=1, tile_y=6, zchunk=5, graph=0), fields=f)
    two = run_gpu(rd, cfg, 9, tuning=dict(tsteps=2, tile_y=6, zchunk=5, graph=0), fields=f)
    assert rel_err(one, ref) <= TOL_NONLIN
    assert np.array_equal(one.view(np.uint32), two.view(np.uint32))


def test_odd_tile_height_leftover_step(rd, orc):
    # 2 and 3 steps per launch with odd tile heights leave a one-step launch
    # at the end of the call; the one-step kernel needs an even height, so
    # that launch runs the multi-level kernel at T = 1 (same bits)
    cfg = W.air((70, 15, 11), src=(9, 4, 3))
    f = W.initial_fields(cfg)
    ref = orc.run(cfg, f, 7)
    even = run_gpu(rd, cfg, 7, tuning=dict(tsteps=1, tile_y=6, zchunk=4), fields=f)
    assert rel_err(even, ref) <= TOL_NONLIN
    for t in (dict(tsteps=2, tile_y=5, zchunk=4, graph=0), dict(tsteps=3, tile_y=3, zchunk=5, graph=1)):
        got = run_gpu(rd, cfg, 7, tuning=t, fields=f)
        assert np.array_equal(got.view(np.uint32), even.view(np.uint32)), t


def test_graph_replay_matches_plain_launches(rd):
    cfg = W.brusselator(shape=(48, 40, 36))
    f = W.initial_fields(cfg)
    t = dict(tsteps=1, tile_q=16, tile_y=8, zchunk=12)
    a = run_gpu(rd, cfg, 70, tuning=dict(t, graph=1), fields=f)
    b = run_gpu(rd, cfg, 70, tuning=dict(t, graph=0), fields=f)
    assert np.array_equal(a, b)


def test_steps_split_across_calls_match_one_call(rd):
    cfg = W.air((40, 24, 16), src=(3, 4, 5))
    f = W.initial_fields(cfg)
    with rd.Sim(cfg, tuning=dict(tsteps=2, tile_y=8)) as sim:
        sim.set_fields(f)
        for n in (1, 5, 2, 17, 0, 3):
            sim.step(n)
        a = sim.get_fields()
        assert sim.steps_done == 28
    b = run_gpu(rd, cfg, 28, tuning=dict(tsteps=3, tile_y=4), fields=f)
    assert np.array_equal(a, b)


def test_checkpoint_resume_is_bitwise(rd):
    cfg = W.ch_front(shape=(30, 26, 20))
    f = W.initial_fields(cfg)
    with rd.Sim(cfg) as sim:
        sim.set_fields(f)
        sim.step(9)
        mid = sim.get_fields()
        sim.step(11)
        full = sim.get_fields()
    with rd.Sim(cfg) as sim:
        sim.set_fields(mid)
        sim.step(11)
        resumed = sim.get_fields()
    assert np.array_equal(full, resumed)


@pytest.mark.parametrize("model", ["diffusion", "brusselator", "ch_front", "air", "turing"])
def test_batch_matches_standalone_bitwise(rd, model):
    sizes = [(23, 17, 11), (140, 9, 14), (16, 33, 25), (70, 20, 8)]
    mk = {"diffusion": lambda s, i: W.diffusion_blob(shape=s, seed=i),
          "brusselator": lambda s, i: W.brusselator(shape=s, seed=i),
          "ch_front": lambda s, i: W.ch_front(shape=s, seed=i),
          "air": lambda s, i: W.air(s, src=(1, 2, 3), seed=i),
          "turing": lambda s, i: W.turing(shape=s, seed=i)}[model]
    cfgs = [mk(s, i) for i, s in enumerate(sizes)]
    steps = 15
    tun = dict(tsteps=1, tile_q=16, tile_y=4, zchunk=6, graph=1)
    ref = [run_gpu(rd, c, steps, tuning=tun) for c in cfgs]
    sims = [rd.Sim(c) for c in cfgs]
    for c, s in zip(cfgs, sims):
        s.set_fields(W.initial_fields(c))
    b = rd.Batch(model)
    b.set_tuning(**tun)
    for s in sims:
        b.add(s)
    b.step(7)
    b.step(8)
    b.sync()
    for s, r in zip(sims, ref):
        assert np.array_equal(s.get_fields(), r)
    b.close()
    for s in sims:
        s.close()


def test_batch_members_join_at_different_times(rd):
    a_cfg = W.brusselator(shape=(24, 20, 16), seed=3)
    b_cfg = W.brusselator(shape=(36, 12, 20), seed=4)
    fa, fb = W.initial_fields(a_cfg), W.initial_fields(b_cfg)
    ra = run_gpu(rd, a_cfg, 20, fields=fa)
    rb = run_gpu(rd, b_cfg, 11, fields=fb)
    A, Bs = rd.Sim(a_cfg), rd.Sim(b_cfg)
    A.set_fields(fa)
    Bs.set_fields(fb)
    bt = rd.Batch("brusselator")
    bt.add(A)
    bt.step(9)
    bt.add(Bs)
    bt.step(11)
    bt.sync()
    assert np.array_equal(A.get_fields(), ra)
    assert np.array_equal(Bs.get_fields(), rb)
    bt.close()
    A.close()
    Bs.close()


def test_batch_of_one_with_odd_step_counts(rd):
    # a batch of one steps its member as a single context (graph replays
    # start from level 0); members then join and leave between odd counts
    a_cfg = W.air((40, 18, 22), src=(3, 4, 5), seed=7)
    b_cfg = W.air((70, 10, 13), src=(1, 2, 3), seed=8)
    fa, fb = W.initial_fields(a_cfg), W.initial_fields(b_cfg)
    ra = run_gpu(rd, a_cfg, 57, fields=fa)
    rb = run_gpu(rd, b_cfg, 38, fields=fb)
    A, Bs = rd.Sim(a_cfg), rd.Sim(b_cfg)
    A.set_fields(fa)
    Bs.set_fields(fb)
    bt = rd.Batch("air")
    bt.add(A)
    bt.step(7)
    bt.step(20)
    bt.step(9)
    bt.add(Bs)
    bt.step(21)
    bt.remove(A)
    bt.step(17)
    bt.sync()
    assert np.array_equal(A.get_fields(), ra)
    assert np.array_equal(Bs.get_fields(), rb)
    bt.close()
    A.close()
    Bs.close()


# ------------------------------------------------------------ reductions
def test_mass_reduction_fp64(rd):
    cfg = W.diffusion_blob(shape=(37, 29, 23))
    f = W.initial_fields(cfg)
    with rd.Sim(cfg) as sim:
        sim.set_fields(f)
        s0, q0, bad0 = sim.mass(0)
        assert bad0 == 0
        ref = f[0].astype(np.float64)
        assert abs(s0 - ref.sum()) <= 1e-12 * abs(ref.sum())
        assert abs(q0 - (ref ** 2).sum()) <= 1e-12 * (ref ** 2).sum()
        sim.step(200)
        s1, _, _ = sim.mass(0)
        # zero-flux diffusion conserves mass up to FP32 rounding of the state
        assert abs(s1 - s0) <= 2e-6 * abs(s0)
        again = sim.mass(0)
        assert again[0] == s1      # fixed summation order: bitwise repeatable


def test_mass_counts_nonfinite(rd):
    cfg = W.diffusion_blob(shape=(12, 10, 8))
    f = W.initial_fields(cfg)
    f[0, 3, 4, 5] = np.nan
    f[0, 1, 2, 3] = np.inf
    with rd.Sim(cfg) as sim:
        sim.set_fields(f)
        _, _, bad = sim.mass(0)
        assert bad == 2


# ------------------------------------------------------------ edge cases
def test_smallest_grid(rd, orc):
    for cfg in (W.diffusion_blob(shape=(2, 2, 2)), W.brusselator(shape=(2, 3, 2)),
                W.ch_front(shape=(2, 2, 3)), W.air((3, 2, 2), src=(2, 1, 1))):
        f = W.initial_fields(cfg)
        got = run_gpu(rd, cfg, 5, fields=f)
        assert rel_err(got, orc.run(cfg, f, 5)) <= TOL_NONLIN


def test_zero_steps_is_identity(rd):
    cfg = W.air((9, 8, 7), src=(1, 1, 1))
    f = W.initial_fields(cfg)
    assert np.array_equal(run_gpu(rd, cfg, 0, fields=f), f)


def test_device_pointers_and_torch_memory(rd, orc):
    import torch
    cfg = W.brusselator(shape=(33, 21, 17))
    f = W.initial_fields(cfg)
    ref = orc.run(cfg, f, 12)
    stream = torch.cuda.Stream()
    with rd.Sim(cfg, torch_memory=True, stream=stream) as sim:
        for s in range(2):
            sim.set_field(s, torch.from_numpy(f[s]).cuda())
        sim.step(12)
        out = torch.empty((2,) + f.shape[1:], dtype=torch.float32, device="cuda")
        for s in range(2):
            sim.get_field(s, out[s])
        got = out.cpu().numpy()
    assert rel_err(got, ref) <= TOL_NONLIN


def test_unstable_dt_rejected(rd):
    from paper_1004_0480_gb300 import _lib as L
    with pytest.raises(L.RdError) as e:
        rd.Sim(W.diffusion_blob(8, dt=0.2))
    assert e.value.status == L.RD_EUNSTABLE


def test_oversized_tile_rejected(rd):
    from paper_1004_0480_gb300 import _lib as L
    with rd.Sim(W.ch_front(shape=(300, 300, 8))) as sim:
        with pytest.raises(L.RdError):
            sim.set_tuning(tsteps=2, tile_q=16, tile_y=64)


def test_wait_times_out_without_harm(rd):
    from paper_1004_0480_gb300 import _lib as L
    cfg = W.brusselator(shape=(128, 128, 128))
    with rd.Sim(cfg) as sim:
        sim.set_fields(W.initial_fields(cfg))
        sim.step(400)
        st = sim.wait(0)
        assert st in (L.RD_OK, L.RD_ETIMEOUT)
        assert sim.wait(60000) == L.RD_OK
        assert np.isfinite(sim.get_field(0)).all()


# ------------------------------------------------------------ workloads
def test_diffusion_64_full_run(rd, orc):
    cfg = W.cfg_diffusion_64()
    f = W.initial_fields(cfg)
    ref = orc.run(cfg, f, cfg["steps"])
    got = run_gpu(rd, cfg, cfg["steps"], fields=f)
    assert rel_err(got, ref) <= TOL_DIFF


def test_brusselator_200_steps(rd, orc):
    cfg = W.brusselator(64, steps=200)
    f = W.initial_fields(cfg)
    ref = orc.run(cfg, f, 200)
    for t in (dict(tsteps=1), dict(tsteps=2, tile_y=8), dict(tsteps=3, tile_y=4)):
        assert rel_err(run_gpu(rd, cfg, 200, tuning=t, fields=f), ref) <= TOL_NONLIN


def test_ch_front_200_steps(rd, orc):
    cfg = W.ch_front(48, steps=200)
    f = W.initial_fields(cfg)
    ref = orc.run(cfg, f, 200)
    for t in (dict(tsteps=1, tile_y=8), dict(tsteps=2, tile_y=8)):
        assert rel_err(run_gpu(rd, cfg, 200, tuning=t, fields=f), ref) <= TOL_NONLIN


def test_air_200_steps(rd, orc):
    cfg = W.air((96, 96, 32), src=(20, 48, 2))
    f = W.initial_fields(cfg)
    ref = orc.run(cfg, f, 200)
    assert rel_err(run_gpu(rd, cfg, 200, fields=f), ref) <= TOL_NONLIN


def test_turing_table1_200_steps(rd, orc):
    # the activator-inhibitor system with the paper's Table 1 parameters
    for stencil in (7, 19):
        cfg = W.turing(shape=(48, 40, 36), stencil=stencil)
        f = W.initial_fields(cfg)
        ref = orc.run(cfg, f, 200)
        assert rel_err(run_gpu(rd, cfg, 200, fields=f), ref) <= TOL_NONLIN


def test_brusselator_256_full_size_few_steps(rd, orc):
    cfg = W.cfg_brusselator_256()
    f = W.initial_fields(cfg)
    ref = orc.run(cfg, f, 3)
    with rd.Sim(cfg) as sim:
        sim.autotune()
        sim.set_fields(f)
        sim.step(3)
        got = sim.get_fields()
    assert rel_err(got, ref) <= TOL_NONLIN


def test_air_512_full_size_few_steps(rd, orc):
    cfg = W.cfg_air_512()
    f = W.initial_fields(cfg)
    ref = orc.run(cfg, f, 2)
    got = run_gpu(rd, cfg, 2, fields=f)
    assert rel_err(got, ref) <= TOL_NONLIN


def test_ch_batch_full_sizes(rd, orc):
    cfgs = W.cfg_ch_front_batch()
    sims = [rd.Sim(c) for c in cfgs]
    fields = [W.initial_fields(c) for c in cfgs]
    for s, f in zip(sims, fields):
        s.set_fields(f)
    b = rd.Batch("ch_front")
    for s in sims:
        b.add(s)
    b.step(2)
    b.sync()
    order = np.argsort([c["shape"][0] for c in cfgs])
    for i in list(order[:3]) + [int(order[-1])]:
        ref = orc.run(cfgs[i], fields[i], 2)
        assert rel_err(sims[i].get_fields(), ref) <= TOL_NONLIN
    b.close()
    for s in sims:
        s.close()


def test_long_runs_stay_finite(rd):
    cfg = W.cfg_brusselator_256()
    with rd.Sim(cfg) as sim:
        sim.set_fields(W.initial_fields(cfg))
        sim.step(cfg["steps"])
        for s in range(2):
            tot, sq, bad = sim.mass(s)
            assert bad == 0 and np.isfinite(tot)
        u = sim.get_field(0)
        assert u.min() > 0.0
    cfg = W.cfg_air_512()
    with rd.Sim(cfg) as sim:
        sim.set_fields(W.initial_fields(cfg))
        sim.step(cfg["steps"])
        for s in range(3):
            assert sim.mass(s)[2] == 0
            assert sim.get_field(s).min() >= -1e-6
