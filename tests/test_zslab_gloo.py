"""Z-slab decomposition of one problem over 2 and 3 CPU ranks (gloo): each
rank steps its slab with the FP64 oracle and exchanges ghost planes after
every step; the owned planes of all ranks must equal the undivided oracle
result bit for bit (same neighbours, same arithmetic per cell)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1004_0480_gb300 import workloads as W
from paper_1004_0480_gb300 import zslab as Z


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _cases():
    per_b = W.brusselator(shape=(9, 7, 13))                       # periodic z: a ring
    neu_b = W.brusselator(shape=(10, 6, 11), bc="neumann")
    front = W.ch_front(shape=(8, 7, 14))                          # halo 2, a held at z = 0
    air = W.air((9, 8, 12), src=(4, 3, 6))                        # source inside a middle slab
    air["wind"] = dict(kind="const", u0=0.7)
    air["bc"][0][5] = "dirichlet"                                 # held NO layer on top
    air["bc_value"] = [[0.0] * 5 + [0.05], [0.0] * 6, [0.0] * 6]
    tur19 = W.turing(shape=(8, 9, 10), sigma=0.3, stencil=19)
    per19 = W.with_(W.brusselator(shape=(8, 6, 12)), stencil=19)
    return {"brusselator_periodic": per_b, "brusselator_neumann": neu_b,
            "ch_front": front, "air_const_wind_held_top": air,
            "turing_19pt": tur19, "brusselator_19pt_periodic": per19}


CASES = _cases()
STEPS = 7


def _rank(rank, ws, port, names, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    import oracle
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        for name in names:
            cfg = CASES[name]
            p = Z.plan(cfg, ws, rank)
            f = Z.scatter(W.initial_fields(cfg).astype(np.float64), p)
            f = Z.run(f, p, STEPS, lambda g, n, c=p.cfg: oracle.run(c, g, n), dist, torch)
            out[(name, rank)] = (p.z0, p.z1, np.array(Z.owned(f, p)))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(240)
@pytest.mark.parametrize("ws", [2, 3])
def test_slabs_equal_the_undivided_grid(orc, ws):
    names = sorted(CASES)
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, ws, port, names, out)) for r in range(ws)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(200)
            assert p.exitcode == 0
        res = dict(out)
    for name in names:
        cfg = CASES[name]
        ref = orc.run(cfg, W.initial_fields(cfg).astype(np.float64), STEPS)
        got = np.empty_like(ref)
        covered = 0
        for r in range(ws):
            z0, z1, f = res[(name, r)]
            got[:, z0:z1] = f
            covered += z1 - z0
        assert covered == cfg["shape"][2]
        assert np.array_equal(got, ref), name


def test_split_and_plan_host_logic():
    assert Z.split(10, 3) == [(0, 4), (4, 7), (7, 10)]
    with pytest.raises(ValueError):
        Z.split(2, 3)
    front = W.ch_front(shape=(8, 8, 6))
    p = Z.plan(front, 3, 1)
    assert (p.lo, p.hi, p.lo_peer, p.hi_peer) == (2, 2, 0, 2)
    assert p.cfg["shape"] == (8, 8, 2 + 4)
    p0 = Z.plan(front, 3, 0)
    assert (p0.lo, p0.lo_peer) == (0, None)
    assert p0.cfg["bc"][0][4] == "dirichlet"       # the held layer stays on rank 0
    per = W.brusselator(shape=(8, 8, 8))
    q = Z.plan(per, 2, 0)
    assert (q.lo_peer, q.hi_peer, q.lo, q.hi) == (1, 1, 1, 1)
    assert q.cfg["bc"][0][4] == q.cfg["bc"][0][5] == "neumann"
    with pytest.raises(ValueError):
        Z.plan(W.air((8, 8, 8), src=(1, 1, 1)), 2, 0)  # logarithmic wind
    with pytest.raises(ValueError):
        Z.plan(W.ch_front(shape=(8, 8, 5)), 3, 0)      # a slab thinner than the halo


def _rank_moments(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    import oracle
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        cfg = CASES["ch_front"]
        p = Z.plan(cfg, ws, rank)
        slab = Z.HostSlab(Z.scatter(W.initial_fields(cfg).astype(np.float64), p),
                          lambda g, n, c=p.cfg: oracle.run(c, g, n), p)
        Z.run_slab(slab, p, STEPS, dist)
        out[rank] = [Z.owned_moments(slab, s, dist).numpy() for s in range(3)]
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(240)
def test_owned_moments_are_all_reduced_in_fp64(orc):
    # every rank ends with the whole grid's moments: the FP64 sums of its
    # owned planes, added over the ranks by an all-reduce
    ws = 3
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank_moments, args=(r, ws, port, out)) for r in range(ws)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(200)
            assert p.exitcode == 0
        res = dict(out)
    cfg = CASES["ch_front"]
    ref = orc.run(cfg, W.initial_fields(cfg).astype(np.float64), STEPS)
    for s in range(3):
        want = np.array([ref[s].sum(), (ref[s] ** 2).sum(), 0.0])
        for r in range(ws):
            np.testing.assert_allclose(res[r][s], want, rtol=1e-12, atol=1e-12)


def test_messages_pair_up():
    # every send has the matching receive on its peer (same tag, same size)
    for cfg in CASES.values():
        for ws in (2, 3, 4):
            try:
                plans = [Z.plan(cfg, ws, r) for r in range(ws)]
            except ValueError:
                continue
            sends = {(r, peer, tag): k for r, p in enumerate(plans)
                     for peer, tag, _, k in Z.messages(p)[0]}
            recvs = {(peer, r, tag): k for r, p in enumerate(plans)
                     for peer, tag, _, k in Z.messages(p)[1]}
            assert sends == recvs


def test_messages_match_in_posting_order_without_tags():
    # NCCL pairs the messages between two ranks by the order they are posted
    # and ignores tags: the k-th send from A to B must be the k-th receive
    # on B from A, for every pair, with the same tag and size
    def pairs(order):
        bad = 0
        for cfg in CASES.values():
            for ws in (2, 3, 4):
                try:
                    plans = [Z.plan(cfg, ws, r) for r in range(ws)]
                except ValueError:
                    continue
                for a in range(ws):
                    for b in range(ws):
                        out = [(t, k) for peer, t, _, k in order(plans[a])[0] if peer == b]
                        inc = [(t, k) for peer, t, _, k in order(plans[b])[1] if peer == a]
                        assert len(out) == len(inc)
                        bad += out != inc
        return bad

    assert pairs(Z.posting_order) == 0
    # the order messages() lists them in would cross the two messages of a
    # periodic two-rank split (a rank's lowest planes landing in the
    # other's lower ghost planes)
    assert pairs(Z.messages) > 0
