"""The resident step kernel (RD_KERNEL_RESIDENT: many steps per cooperative
launch; tiles advanced K steps per round in shared memory from a halo of K,
a grid-wide barrier between rounds) through the C ABI.

It evaluates the march kernel's per-cell arithmetic on the same neighbour
values and rounds every level to the state's type, so it must agree with
the one-step march kernel bit for bit, for every model it takes, both
storage types, ragged and periodic widths, held layers, the point source and
the wind, and every plan: K = 1..4, tiles of one row up to the whole grid,
last tiles that pass the grid's end, halos wider than a periodic axis.
Against the FP64 oracle the bounds of test_gpu_parity hold (1e-5 pure
diffusion, 1e-4 nonlinear, FP32); the 64^3 inert-diffusion workload runs its
full 100 steps.  The barrier's bounded wait is made to run out with the
phantom-CTA hook: the launch stops, rd_sync reports RD_ETIMEOUT, and the
context stays usable.
"""
import numpy as np
import pytest

from paper_1004_0480_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_DIFF = 1e-5
TOL_NONLIN = 1e-4
MARCH = dict(tsteps=1, tile_q=16, tile_y=6, zchunk=5, graph=0)
# forced plans (K, tile_y, tile_z); one whose rows and halo do not fit
# shared memory for a problem is refused with RD_EINVAL and skipped there
PLANS = [(1, 0, 0), (2, 1, 1), (3, 1, 2), (4, 1, 1), (3, 2, 3), (4, 5, 2), (4, 64, 64)]


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


def run_gpu(rd, cfg, steps, kernel, storage="f32", fields=None, chunks=None, plan=None):
    """Fields after ``steps`` steps; None when ``plan`` does not fit."""
    from paper_1004_0480_gb300 import _lib as L
    f = W.initial_fields(cfg) if fields is None else fields
    with rd.Sim(cfg, storage) as sim:
        if kernel == "march":
            sim.set_tuning(**MARCH)
        else:
            sim.set_kernel(kernel)
            if plan:
                try:
                    sim.set_resident_plan(*plan)
                except L.RdError as e:
                    if e.status != L.RD_EINVAL:
                        raise
                    return None
        sim.set_fields(f)
        for k in (chunks or [steps]):
            sim.step(k)
        sim.sync()
        return sim.get_fields()


def cases():
    out = {}
    for nx in (64, 65, 66, 67, 3, 16, 141):
        out[f"diffusion_neumann_{nx}"] = (W.diffusion_blob(shape=(nx, 23, 19)), TOL_DIFF)
    per_d = W.diffusion_blob(shape=(67, 23, 19))
    per_d["bc"] = [["periodic"] * 6]
    out["diffusion_periodic_67"] = (per_d, TOL_DIFF)
    per_d = W.diffusion_blob(shape=(132, 9, 4))
    per_d["bc"] = [["periodic"] * 6]
    out["diffusion_periodic_132"] = (per_d, TOL_DIFF)
    aniso = W.diffusion_blob(shape=(141, 24, 19))
    aniso["D"] = [[0.9, 0.3, 0.05]]
    aniso["dt"] = 0.4
    out["diffusion_anisotropic"] = (aniso, TOL_DIFF)
    out["brusselator_periodic_70"] = (W.brusselator(shape=(70, 20, 17)), TOL_NONLIN)
    out["brusselator_neumann"] = (W.brusselator(shape=(141, 23, 19), bc="neumann"), TOL_NONLIN)
    out["air_neumann"] = (W.air((141, 23, 19), src=(5, 17, 2)), TOL_NONLIN)
    air_per = W.air((133, 24, 19), src=(130, 0, 17))
    air_per["bc"] = [["periodic"] * 6 for _ in range(3)]
    out["air_periodic_133"] = (air_per, TOL_NONLIN)
    air_held = W.air((67, 24, 19), src=(66, 23, 5))
    air_held["bc"] = [["neumann", "dirichlet", "neumann", "neumann", "periodic", "periodic"]] * 3
    air_held["bc_value"] = [[0.0, v, 0.0, 0.0, 0.0, 0.0] for v in (0.0, 0.02, 1.0)]
    air_held["wind"] = dict(kind="const", u0=-0.5)
    out["air_held_reverse_wind_67"] = (air_held, TOL_NONLIN)
    held_all = W.diffusion_blob(shape=(37, 21, 13))
    held_all["bc"] = [["dirichlet"] * 6]
    held_all["bc_value"] = [[0.1, 0.2, 0.3, 0.4, 0.5, 0.6]]
    out["diffusion_held_every_face"] = (held_all, TOL_DIFF)
    out["turing"] = (W.turing(shape=(141, 23, 19), sigma=0.3), TOL_NONLIN)
    out["diffusion_2cube"] = (W.diffusion_blob(shape=(2, 2, 2)), TOL_DIFF)
    out["air_3x2x2"] = (W.air((3, 2, 2), src=(2, 1, 1)), TOL_NONLIN)
    per_small = W.brusselator(shape=(9, 3, 2))
    out["brusselator_periodic_9x3x2"] = (per_small, TOL_NONLIN)
    mixed = W.diffusion_blob(shape=(30, 7, 11))
    mixed["bc"] = [["neumann", "neumann", "periodic", "periodic", "neumann", "neumann"]]
    out["diffusion_periodic_y_only"] = (mixed, TOL_DIFF)
    return out


CASES = cases()


@pytest.mark.parametrize("name", sorted(CASES))
def test_resident_equals_march_and_the_oracle(rd, orc, name):
    cfg, tol = CASES[name]
    f = W.initial_fields(cfg)
    for steps in (1, 2, 13):
        march = run_gpu(rd, cfg, steps, "march", fields=f)
        got = run_gpu(rd, cfg, steps, "resident", fields=f)
        assert np.array_equal(got.view(np.uint32), march.view(np.uint32)), \
            f"{name}: {steps} steps differ from the march kernel"
    ran = 0
    for plan in PLANS:
        got = run_gpu(rd, cfg, 13, "resident", fields=f, plan=plan)
        if got is None:
            continue
        ran += 1
        assert np.array_equal(got.view(np.uint32), march.view(np.uint32)), \
            f"{name}: plan {plan} differs from the march kernel"
    assert ran >= 3
    ref = orc.run(cfg, f, 13)
    assert rel_err(march, ref) <= tol


@pytest.mark.parametrize("name", ["brusselator_periodic_70", "air_neumann",
                                  "diffusion_neumann_67", "diffusion_held_every_face"])
def test_resident_bf16_equals_march(rd, name):
    cfg, _ = CASES[name]
    f = W.initial_fields(cfg)
    march = run_gpu(rd, cfg, 11, "march", storage="bf16", fields=f)
    for plan in [None] + PLANS:
        got = run_gpu(rd, cfg, 11, "resident", storage="bf16", fields=f, plan=plan)
        if got is not None:
            assert np.array_equal(got.view(np.uint32), march.view(np.uint32)), plan


def test_resident_diffusion_64_full_run(rd, orc):
    cfg = W.cfg_diffusion_64()
    f = W.initial_fields(cfg)
    ref = orc.run(cfg, f, cfg["steps"])
    got = run_gpu(rd, cfg, cfg["steps"], "resident", fields=f)
    assert rel_err(got, ref) <= TOL_DIFF
    march = run_gpu(rd, cfg, cfg["steps"], "march", fields=f)
    assert np.array_equal(got.view(np.uint32), march.view(np.uint32))
    for plan in PLANS:
        got = run_gpu(rd, cfg, cfg["steps"], "resident", fields=f, plan=plan)
        if got is not None:
            assert np.array_equal(got.view(np.uint32), march.view(np.uint32)), plan


def test_resident_many_calls_and_a_split_launch(rd):
    # 65 536 steps is one launch's limit: 65 541 steps take two launches;
    # odd and even chunks leave the state in either level
    cfg = W.diffusion_blob(shape=(12, 8, 8))
    cfg["bc"] = [["periodic"] * 6]
    f = W.initial_fields(cfg)
    march = run_gpu(rd, cfg, 65541, "march", fields=f)
    got = run_gpu(rd, cfg, 65541, "resident", fields=f)
    assert np.array_equal(got, march)
    got = run_gpu(rd, cfg, 65541, "resident", fields=f, chunks=[1, 2, 3, 65535])
    assert np.array_equal(got, march)
    got = run_gpu(rd, cfg, 65541, "resident", fields=f, chunks=[5, 7, 65529], plan=(3, 2, 3))
    assert got is not None and np.array_equal(got, march)
    with rd.Sim(cfg) as sim:
        sim.set_kernel("resident")
        sim.set_fields(f)
        before = sim.launches
        sim.step(65541)
        sim.sync()
        assert sim.launches - before == 2
        assert sim.steps_done == 65541


def test_resident_refusals(rd):
    from paper_1004_0480_gb300 import _lib as L
    refused = [W.with_(W.brusselator(shape=(32, 16, 8)), stencil=19),
               W.ch_front(shape=(32, 16, 8)),
               W.ch_table1(shape=(32, 16, 8)),
               W.plume(shape=(32, 16, 8), src=(3, 3, 3))]
    for cfg in refused:
        with rd.Sim(cfg) as sim:
            with pytest.raises(L.RdError) as e:
                sim.set_kernel("resident")
            assert e.value.status == L.RD_EUNSUPPORTED, cfg["model"]
            assert sim.kernel == "march"
    # rows too wide for shared memory even in a one-row tile
    with rd.Sim(W.diffusion_blob(shape=(65536, 2, 2))) as sim:
        with pytest.raises(L.RdError) as e:
            sim.set_kernel("resident")
        assert e.value.status == L.RD_EUNSUPPORTED
    with rd.Sim(W.diffusion_blob(shape=(32, 16, 8))) as sim:
        with pytest.raises(L.RdError) as e:
            sim.set_resident_plan(2, 1, 1)           # not the resident kernel
        assert e.value.status == L.RD_EUNSUPPORTED
        sim.set_kernel("resident")
        assert sim.kernel == "resident"
        plan = sim.resident_plan()
        assert 1 <= plan["K"] <= 4 and plan["ctas"] <= plan["tiles"]
        for bad in ((5, 0, 0), (-1, 0, 0), (1, -1, 0), (1, 0, -2)):
            with pytest.raises(L.RdError) as e:
                sim.set_resident_plan(*bad)
            assert e.value.status == L.RD_EINVAL, bad
            assert sim.resident_plan() == plan          # the previous plan stays
        sim.set_resident_plan(3, 100, 5)             # tile clamped to the grid
        got = sim.resident_plan()
        assert (got["K"], got["tile_y"], got["tile_z"], got["tiles"]) == (3, 16, 5, 2)
    with rd.Sim(W.diffusion_blob(shape=(4096, 64, 8))) as sim:
        sim.set_kernel("resident")
        with pytest.raises(L.RdError) as e:
            sim.set_resident_plan(4, 64, 8)          # 72 x 16 rows of 16 KiB
        assert e.value.status == L.RD_EINVAL
        with pytest.raises(L.RdError) as e:
            sim.autotune()
        assert e.value.status == L.RD_EUNSUPPORTED
        sim.set_kernel("march")
        assert sim.lib.rd_debug_resident_stall(sim.ctx, 1) == L.RD_EUNSUPPORTED


def test_resident_barrier_timeout_is_reported_and_the_context_recovers(rd):
    from paper_1004_0480_gb300 import _lib as L
    cfg = W.diffusion_blob(shape=(40, 24, 16))
    f = W.initial_fields(cfg)
    march = run_gpu(rd, cfg, 6, "march", fields=f)
    with rd.Sim(cfg) as sim:
        sim.set_kernel("resident")
        sim.set_fields(f)
        assert sim.lib.rd_debug_resident_stall(sim.ctx, -1) == L.RD_EINVAL
        # one CTA that never arrives: the first barrier wait runs out
        sim.set_resident_plan(2, 0, 0)
        assert sim.lib.rd_debug_resident_stall(sim.ctx, 1) == L.RD_OK
        sim.step(2)                                  # one round: no barrier, hook kept
        sim.sync()
        sim.step(5)
        with pytest.raises(L.RdError) as e:
            sim.sync()
        assert e.value.status == L.RD_ETIMEOUT
        # reported once; the next launches run normally
        sim.sync()
        sim.set_fields(f)
        sim.step(6)
        sim.sync()
        assert np.array_equal(sim.get_fields(), march)


def test_resident_tile_copies_by_tensor_memory_where_no_box_wraps(rd):
    """Tiles arrive as one tensor-memory box unless y or z is periodic (a
    box cannot wrap) or rows exceed 256 elements; both paths are covered by
    the bit-for-bit comparisons above (zero-flux cases take boxes, the
    periodic ones per-thread copies)."""
    per_x = W.diffusion_blob(shape=(40, 12, 10))
    per_x["bc"] = [["periodic", "periodic", "neumann", "neumann", "neumann", "neumann"]]
    per_z = W.diffusion_blob(shape=(40, 12, 10))
    per_z["bc"] = [["neumann", "neumann", "neumann", "neumann", "periodic", "periodic"]]
    expect = [(W.cfg_diffusion_64(), 1), (per_x, 1), (per_z, 0),
              (W.brusselator(shape=(70, 20, 17)), 0),          # periodic on every axis
              (W.diffusion_blob(shape=(256, 6, 6)), 1),         # a box of 256 elements
              (W.diffusion_blob(shape=(260, 6, 6)), 0),         # rows wider than 256
              (W.diffusion_blob(shape=(300, 6, 6)), 0)]
    for cfg, tma in expect:
        with rd.Sim(cfg) as sim:
            sim.set_kernel("resident")
            assert sim.resident_plan()["tma"] == tma, cfg["name"]
    f = W.initial_fields(per_x)
    march = run_gpu(rd, per_x, 9, "march", fields=f)
    for plan in (None, (3, 5, 2), (1, 12, 10)):
        got = run_gpu(rd, per_x, 9, "resident", fields=f, plan=plan)
        assert np.array_equal(got.view(np.uint32), march.view(np.uint32)), plan
    for shape in ((300, 6, 6), (256, 6, 6), (253, 7, 5)):
        cfg = W.diffusion_blob(shape=shape)
        f = W.initial_fields(cfg)
        march = run_gpu(rd, cfg, 7, "march", fields=f)
        got = run_gpu(rd, cfg, 7, "resident", fields=f)
        assert np.array_equal(got.view(np.uint32), march.view(np.uint32)), shape
