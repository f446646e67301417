"""The paper's Shared and Moving Tiles kernel designs (Section 4.1, Tables
4-5), restated for this GPU as ablation baselines of the 19-point step:
against the FP64 oracle and against the march kernel, through the C ABI.

Tolerances as in ``test_gpu_parity`` (normwise max relative error 1e-5 for
pure diffusion, 1e-4 for the nonlinear problems, FP32 state).  The designs
sum the stencil in another order than the march kernel, so they agree with
it to rounding, not bit for bit.
"""
import numpy as np
import pytest

from paper_1004_0480_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_DIFF = 1e-5
TOL_NONLIN = 1e-4
SHAPE = (141, 23, 19)   # ragged in every tile dimension of both designs
KERNELS = ["shared", "tiles"]


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


def run(rd, cfg, steps, kernel, fields, graph=0):
    with rd.Sim(cfg) as sim:
        sim.set_tuning(graph=graph)
        sim.set_kernel(kernel)
        assert sim.kernel == kernel
        sim.set_fields(fields)
        sim.step(steps)
        return sim.get_fields()


def s19(cfg, **kw):
    return W.with_(cfg, stencil=19, **kw)


def cases():
    per_d = s19(W.diffusion_blob(shape=SHAPE))
    per_d["bc"] = [["periodic"] * 6]
    mixed_b = s19(W.brusselator(shape=SHAPE))
    mixed_b["bc"] = [["neumann", "neumann", "periodic", "periodic", "neumann", "neumann"]] * 2
    air = s19(W.air(SHAPE, src=(0, 0, 0)), D=[[0.1] * 3] * 3, wind=None, source=None)
    return {
        "diffusion_neumann": (s19(W.diffusion_blob(shape=SHAPE)), TOL_DIFF),
        "diffusion_periodic": (per_d, TOL_DIFF),
        "brusselator_periodic": (s19(W.brusselator(shape=SHAPE)), TOL_NONLIN),
        "brusselator_mixed_bc": (mixed_b, TOL_NONLIN),
        "air_no_wind": (air, TOL_NONLIN),
        "brusselator_tiny_periodic": (s19(W.brusselator(shape=(5, 3, 7))), TOL_NONLIN),
        "brusselator_2cube_neumann": (s19(W.brusselator(shape=(2, 2, 2), bc="neumann")),
                                      TOL_NONLIN),
    }


CASES = cases()


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("name", sorted(CASES))
def test_paper_design_matches_oracle_and_march_kernel(rd, orc, kernel, name):
    cfg, tol = CASES[name]
    steps = 13
    f = W.initial_fields(cfg)
    ref = orc.run(cfg, f, steps)
    got = run(rd, cfg, steps, kernel, f)
    assert rel_err(got, ref) <= tol, f"{kernel} {name}"
    march = run(rd, cfg, steps, "march", f)
    assert rel_err(got, march) <= tol


@pytest.mark.parametrize("kernel", KERNELS)
def test_paper_design_graph_replay(rd, kernel):
    cfg = s19(W.brusselator(shape=(96, 40, 24)))
    f = W.initial_fields(cfg)
    a = run(rd, cfg, 40, kernel, f, graph=0)
    b = run(rd, cfg, 40, kernel, f, graph=1)
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_paper_designs_are_refused_where_undefined(rd):
    from paper_1004_0480_gb300 import _lib as L
    refused = [W.brusselator(shape=(64, 8, 8)),                       # 7-point stencil
               s19(W.air((64, 8, 8), src=(1, 1, 1)), D=[[0.1] * 3] * 3)]  # wind and source
    for cfg in refused:
        with rd.Sim(cfg) as sim:
            assert sim.lib.rd_set_kernel(sim.ctx, L.KERNEL["shared"]) == L.RD_EUNSUPPORTED
            assert sim.kernel == "march"
    with rd.Sim(s19(W.brusselator(shape=(64, 8, 8))), storage="bf16") as sim:
        assert sim.lib.rd_set_kernel(sim.ctx, L.KERNEL["tiles"]) == L.RD_EUNSUPPORTED
    with rd.Sim(s19(W.brusselator(shape=(64, 8, 8)))) as sim:
        assert sim.lib.rd_set_kernel(sim.ctx, 7) == L.RD_EINVAL
        sim.set_kernel("tiles")
        with pytest.raises(Exception):
            sim.autotune()                  # the autotuner tunes the march kernel only
        sim.set_kernel("march")
        sim.autotune()
