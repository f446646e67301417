"""Served results equal the same requests run alone (the plain stepper),
bit for bit: batching, admission order and neighbours in the mix do not
change any request's arithmetic."""
import numpy as np
import pytest

from paper_1004_0480_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def serving():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1004_0480_gb300 import build as B
    B.build()
    from paper_1004_0480_gb300 import serving
    return serving


@pytest.mark.parametrize("run_cells", [float("inf"), 60_000])
def test_mix_equals_alone(serving, run_cells):
    # run_cells 60 000: requests join running batches one after another
    specs = W.serving_requests(count=10, rate_per_s=400.0, seed=11, edges=(24, 33, 48, 64),
                               steps_lo=10, steps_hi=90)
    reqs = serving.requests_from_workload(specs)
    eng = serving.CudaEngine()
    res, st = serving.Server(eng, budget_bytes=2e9, quantum=13,
                             run_cells=run_cells).run(reqs, collect_fields=True)
    eng.shutdown()
    alone, _ = serving.serve_plain(serving.CudaEngine(), reqs, collect_fields=True)
    by_id = {r.id: r for r in alone}
    assert len(res) == len(reqs) == len(alone)
    for r in res:
        a = by_id[r.id]
        assert r.fields.shape == a.fields.shape
        assert np.array_equal(r.fields, a.fields), f"request {r.id} differs in the mix"
    assert st.p50 <= st.p99


def test_served_requests_match_the_oracle(serving, orc):
    specs = W.serving_requests(count=4, rate_per_s=1000.0, seed=12, edges=(20, 28),
                               steps_lo=15, steps_hi=40)
    reqs = serving.requests_from_workload(specs)
    eng = serving.CudaEngine()
    res, _ = serving.Server(eng, budget_bytes=1e9, quantum=9).run(reqs, collect_fields=True)
    eng.shutdown()
    cfgs = {r.id: r.cfg for r in reqs}
    for r in res:
        cfg = cfgs[r.id]
        ref = orc.run(cfg, W.initial_fields(cfg), r.steps)
        tol = 1e-5 if cfg["model"] == "diffusion" else 1e-4
        err = max(float(np.abs(r.fields[s] - ref[s]).max() / np.abs(ref[s]).max())
                  for s in range(cfg["nspecies"]))
        assert err <= tol
