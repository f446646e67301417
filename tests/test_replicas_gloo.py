"""The N > 1 path of bench.py on two CPU ranks (gloo): each rank is an
independent replica; the only cross-rank work is the barrier and the
max-over-ranks reduction of the timed region, and the whole-job value counts
every rank's cell-steps over the slowest rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(ws),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    import torch.distributed as dist
    w, r, _ = bench.dist_setup(ws)
    assert (w, r) == (ws, rank)
    assert dist.get_backend() == "gloo"
    bench.barrier(w)
    elapsed = 1.0 + rank          # rank 1 is the slow replica
    slowest = bench.max_over_ranks(elapsed, w)
    out[rank] = (slowest, bench.whole_job_glups(3e9, w, slowest))
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_replicas():
    ws = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, ws, port, out)) for r in range(ws)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(100)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0] == res[1]
    slowest, value = res[0]
    assert slowest == 2.0
    assert value == pytest.approx(3e9 * 2 / 2.0 / 1e9)
