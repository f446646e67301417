"""rd_batch_step_each: the members of a batch advance their own step counts
in one batched launch sequence (members whose count is used up are left
alone), through the C ABI.

Every member must equal the same problem stepped alone by its count, bit
for bit: batches and single contexts evaluate the same per-cell code, and
a member left alone keeps the level its last step wrote.  Cases: counts
across graph replays (16 launches per batch graph) and remainders, a zero
count, two calls in a row, the 19-point Cahn-Hilliard model (two launches
per step), the plume (its step counter stops with the member and resumes),
and the refusal of more than one step per launch.
"""
import numpy as np
import pytest

from paper_1004_0480_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1004_0480_gb300 import build as B
    B.build()
    from paper_1004_0480_gb300 import sim
    return sim


def alone(rd, cfg, steps, fields):
    with rd.Sim(cfg) as sim:
        sim.set_fields(fields)
        sim.step(steps)
        sim.sync()
        return sim.get_fields()


def run_each(rd, model, cfgs, calls, tuning):
    """Batch of ``cfgs``; ``calls``: per-call lists of member counts."""
    fields = [W.initial_fields(c) for c in cfgs]
    sims = [rd.Sim(c) for c in cfgs]
    try:
        for s, f in zip(sims, fields):
            s.set_fields(f)
        b = rd.Batch(model)
        b.set_tuning(**tuning)
        for s in sims:
            b.add(s)
        for counts in calls:
            b.step_each(dict(zip(sims, counts)))
        b.sync()
        got = [s.get_fields() for s in sims]
        done = [s.steps_done for s in sims]
        b.close()
    finally:
        for s in sims:
            s.close()
    return fields, got, done


def check(rd, cfgs, fields, got, done, calls):
    for i, cfg in enumerate(cfgs):
        n = sum(c[i] for c in calls)
        assert done[i] == n
        ref = alone(rd, cfg, n, fields[i]) if n else fields[i]
        assert np.array_equal(got[i].view(np.uint32), ref.view(np.uint32)), \
            f"member {i} ({cfg['shape']}, {n} steps)"


def test_members_advance_their_own_counts(rd):
    sizes = [(23, 17, 11), (70, 9, 14), (16, 33, 9), (41, 20, 12)]
    cfgs = [W.brusselator(shape=s, seed=i) for i, s in enumerate(sizes)]
    calls = [[0, 5, 17, 33], [3, 0, 20, 1]]
    tun = dict(tsteps=1, tile_q=16, tile_y=6, zchunk=5, graph=1)
    fields, got, done = run_each(rd, "brusselator", cfgs, calls, tun)
    check(rd, cfgs, fields, got, done, calls)


def test_air_with_wind_and_source_no_graph(rd):
    cfgs = [W.air(s, src=(1, 2, 3), seed=i)
            for i, s in enumerate([(23, 17, 11), (40, 12, 9), (16, 33, 25)])]
    calls = [[9, 2, 5]]
    tun = dict(tsteps=1, tile_q=16, tile_y=4, zchunk=6, graph=0)
    fields, got, done = run_each(rd, "air", cfgs, calls, tun)
    check(rd, cfgs, fields, got, done, calls)


def test_two_launches_per_step_cahn_hilliard_19(rd):
    cfgs = [W.with_(W.ch_table1(shape=s, seed=i), init="uniform_noise")
            for i, s in enumerate([(20, 14, 12), (33, 10, 9)])]
    calls = [[3, 7], [2, 0]]
    tun = dict(tsteps=1, tile_q=16, tile_y=4, zchunk=5, graph=1)
    fields, got, done = run_each(rd, "ch_table1", cfgs, calls, tun)
    check(rd, cfgs, fields, got, done, calls)


def test_plume_step_counter_stops_and_resumes(rd):
    # u_z depends on each member's step index: a member stopped early must
    # resume at its own index in the next call
    cfgs = [W.with_(W.plume(shape=s, src=(5, 4, 3)), stencil=19, init="uniform_noise",
                    seed=i) for i, s in enumerate([(24, 16, 20), (36, 12, 18)])]
    calls = [[4, 19], [8, 3]]
    tun = dict(tsteps=1, tile_q=16, tile_y=4, zchunk=5, graph=1)
    fields, got, done = run_each(rd, "diffusion", cfgs, calls, tun)
    check(rd, cfgs, fields, got, done, calls)


def test_more_than_one_step_per_launch_is_refused(rd):
    from paper_1004_0480_gb300 import _lib as L
    cfgs = [W.brusselator(shape=(23, 17, 11)), W.brusselator(shape=(16, 9, 8))]
    sims = [rd.Sim(c) for c in cfgs]
    try:
        b = rd.Batch("brusselator")
        b.set_tuning(tsteps=2, tile_q=16, tile_y=6, zchunk=5, graph=0)
        for s in sims:
            b.add(s)
        with pytest.raises(L.RdError) as e:
            b.step_each({sims[0]: 4, sims[1]: 2})
        assert e.value.status == L.RD_EINVAL
        with pytest.raises(L.RdError):
            b.step_each({sims[0]: -1})
        b.close()
    finally:
        for s in sims:
            s.close()
