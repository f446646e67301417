"""The one-step 7-point kernel with 8 cells per thread (tile_q = 8: x
neighbours by warp shuffle, 16-byte bfloat16 copies) against the 4-cell
kernel and the FP64 oracle, through the C ABI.

Both kernels evaluate the same per-cell functions in the same order, so they
must agree bit for bit; the oracle bounds are those of test_gpu_parity
(1e-5 pure diffusion, 1e-4 nonlinear, FP32).  Widths cover nx % 8 = 0..7
(vectors straddling a zero-flux face, periodic rows that wrap inside a
vector), tiles whose halo rows are ghost rows, and z-chunks that end inside
and at the end of the march.
"""
import numpy as np
import pytest

from paper_1004_0480_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_DIFF = 1e-5
TOL_NONLIN = 1e-4
FOUR = dict(tsteps=1, tile_q=16, tile_y=6, zchunk=5, graph=0)
WIDE = [
    dict(tsteps=1, tile_q=8, tile_y=4, zchunk=5, graph=0),
    dict(tsteps=1, tile_q=8, tile_y=8, zchunk=19, graph=1),
    dict(tsteps=1, tile_q=8, tile_y=12, zchunk=7, graph=1),
    dict(tsteps=1, tile_q=8, tile_y=16, zchunk=3, graph=0),
]


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


def cases():
    out = {}
    # nx % 8 = 0..7, and zero-flux faces ending a vector at every lane of a
    # tile row (nx % 64 = 8, 16, ..., 56)
    for nx in (64, 65, 66, 67, 68, 69, 70, 71, 141, 16, 24, 40, 72, 80, 104, 120):
        out[f"diffusion_neumann_{nx}"] = (W.diffusion_blob(shape=(nx, 23, 19)), TOL_DIFF)
    per_d = W.diffusion_blob(shape=(132, 23, 19))
    per_d["bc"] = [["periodic"] * 6]
    out["diffusion_periodic_132"] = (per_d, TOL_DIFF)
    aniso = W.diffusion_blob(shape=(141, 24, 19))
    aniso["D"] = [[0.9, 0.3, 0.05]]
    aniso["dt"] = 0.4
    out["diffusion_anisotropic"] = (aniso, TOL_DIFF)
    out["brusselator_periodic_132"] = (W.brusselator(shape=(132, 24, 17)), TOL_NONLIN)
    out["brusselator_periodic_70"] = (W.brusselator(shape=(70, 20, 17)), TOL_NONLIN)
    out["brusselator_neumann"] = (W.brusselator(shape=(141, 23, 19), bc="neumann"), TOL_NONLIN)
    out["brusselator_neumann_48"] = (W.brusselator(shape=(48, 23, 19), bc="neumann"), TOL_NONLIN)
    out["air_neumann_16"] = (W.air((16, 33, 25), src=(1, 2, 3)), TOL_NONLIN)
    out["air_neumann"] = (W.air((141, 23, 19), src=(5, 17, 2)), TOL_NONLIN)
    air_per = W.air((133, 24, 19), src=(130, 0, 17))
    air_per["bc"] = [["periodic"] * 6 for _ in range(3)]
    out["air_periodic_133"] = (air_per, TOL_NONLIN)
    air_held = W.air((67, 24, 19), src=(66, 23, 5))
    air_held["bc"] = [["neumann", "dirichlet", "neumann", "neumann", "periodic", "periodic"]] * 3
    air_held["bc_value"] = [[0.0, v, 0.0, 0.0, 0.0, 0.0] for v in (0.0, 0.02, 1.0)]
    air_held["wind"] = dict(kind="const", u0=-0.5)
    out["air_held_reverse_wind_67"] = (air_held, TOL_NONLIN)
    out["turing"] = (W.turing(shape=(141, 23, 19), sigma=0.3), TOL_NONLIN)
    plume = W.with_(W.plume(shape=(70, 36, 40), src=(20, 18, 9)), init="uniform_noise")
    out["plume_3d_wind"] = (plume, TOL_NONLIN)
    return out


CASES = cases()


@pytest.mark.parametrize("name", sorted(CASES))
def test_wide_kernel_equals_the_four_cell_kernel_and_the_oracle(rd, orc, name):
    cfg, tol = CASES[name]
    steps = 13
    f = W.initial_fields(cfg)
    ref = orc.run(cfg, f, steps)
    four = run_gpu(rd, cfg, steps, tuning=FOUR, fields=f)
    assert rel_err(four, ref) <= tol
    for t in WIDE:
        got = run_gpu(rd, cfg, steps, tuning=t, fields=f)
        assert np.array_equal(got.view(np.uint32), four.view(np.uint32)), \
            f"{name} {t}: differs from the 4-cell kernel"


@pytest.mark.parametrize("name", ["brusselator_periodic_132", "air_neumann",
                                  "diffusion_neumann_67"])
def test_wide_kernel_bf16_equals_the_four_cell_kernel(rd, name):
    cfg, _ = CASES[name]
    f = W.initial_fields(cfg)
    four = run_gpu(rd, cfg, 10, storage="bf16", tuning=FOUR, fields=f)
    for t in WIDE[:2]:
        got = run_gpu(rd, cfg, 10, storage="bf16", tuning=t, fields=f)
        assert np.array_equal(got.view(np.uint32), four.view(np.uint32)), t


def test_wide_kernel_in_batches(rd):
    sizes = [(23, 17, 11), (140, 9, 14), (16, 33, 25), (70, 20, 8)]
    cfgs = [W.air(s, src=(1, 2, 3), seed=i) for i, s in enumerate(sizes)]
    tun = dict(tsteps=1, tile_q=8, tile_y=8, zchunk=6, graph=1)
    ref = [run_gpu(rd, c, 21, tuning=FOUR) for c in cfgs]
    sims = [rd.Sim(c) for c in cfgs]
    try:
        for c, s in zip(cfgs, sims):
            s.set_fields(W.initial_fields(c))
        b = rd.Batch("air")
        b.set_tuning(**tun)
        for s in sims:
            b.add(s)
        b.step(21)
        b.sync()
        for s, r in zip(sims, ref):
            assert np.array_equal(s.get_fields(), r)
        b.close()
    finally:
        for s in sims:
            s.close()


def test_wide_kernel_full_size_brusselator(rd, orc):
    cfg = W.cfg_brusselator_256()
    f = W.initial_fields(cfg)
    ref = orc.run(cfg, f, 2)
    got = run_gpu(rd, cfg, 2, tuning=dict(tsteps=1, tile_q=8, tile_y=16, zchunk=64), fields=f)
    assert rel_err(got, ref) <= TOL_NONLIN


def test_wide_kernel_tuning_rules(rd):
    from paper_1004_0480_gb300 import _lib as L
    with rd.Sim(W.brusselator(shape=(64, 16, 8))) as sim:
        for bad in (dict(tile_q=8, tile_y=6),        # 48 compute threads: a split warp
                    dict(tile_q=8, tile_y=2),
                    dict(tile_q=8, tile_y=44),       # more halo vectors than the halo warp holds
                    dict(tile_q=8, tile_y=8, tsteps=2),
                    dict(tile_q=4, tile_y=8)):
            with pytest.raises(L.RdError) as e:
                sim.set_tuning(**bad)
            assert e.value.status == L.RD_EINVAL, bad
        sim.set_tuning(tile_q=8, tile_y=8, tsteps=1)
    with rd.Sim(W.ch_front(shape=(64, 16, 8))) as sim:
        with pytest.raises(L.RdError):
            sim.set_tuning(tile_q=8, tile_y=8)       # the front model has its own kernel
    with rd.Sim(W.with_(W.brusselator(shape=(64, 16, 8)), stencil=19)) as sim:
        with pytest.raises(L.RdError):
            sim.set_tuning(tile_q=8, tile_y=8)       # 7-point only
