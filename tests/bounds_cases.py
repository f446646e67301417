"""Small problems covering every step-kernel family, stepped through the C
ABI by whichever library variant this process loads (RD_BOUNDS_CHECK=1: the
bounds-checked debug build).  Run as a script, it writes every result and
every synchronisation status to an .npz file, for tests/test_gpu_debug_bounds.py
to compare the two variants.

    python tests/bounds_cases.py OUT.npz
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1004_0480_gb300 import workloads as W  # noqa: E402

SHAPE = (70, 21, 13)         # two x-tiles (ragged), ragged y tiles and z chunks


def cases():
    """name -> (problem, storage, tuning, steps); a tuning with "kernel":
    "resident" selects the resident kernel with the plan under "plan"."""
    per_b = W.brusselator(shape=(67, 18, 11))
    t1 = dict(tsteps=1, tile_y=6, zchunk=5, graph=0)
    out = {
        "diffusion_t1": (W.diffusion_blob(shape=SHAPE), "f32", t1, 6),
        "brusselator_periodic_t1": (per_b, "f32", t1, 6),
        "brusselator_t2_odd": (per_b, "f32", dict(tsteps=2, tile_y=5, zchunk=4), 5),
        "air_t3": (W.air(SHAPE, src=(9, 4, 3)), "f32", dict(tsteps=3, tile_y=3, zchunk=4), 7),
        "air_t1_regcap": (W.air(SHAPE, src=(9, 4, 3)), "f32", dict(t1, regcap=1), 6),
        "air_bf16": (W.air(SHAPE, src=(9, 4, 3)), "bf16", t1, 6),
        "front_t1": (W.ch_front(shape=SHAPE), "f32", dict(tsteps=1, tile_y=5, zchunk=5), 6),
        "front_t2": (W.ch_front(shape=SHAPE), "f32", dict(tsteps=2, tile_y=4, zchunk=6), 6),
        "front_bf16": (W.ch_front(shape=SHAPE), "bf16", dict(tsteps=1, tile_y=4, zchunk=5), 6),
        "brusselator_19": (W.with_(per_b, stencil=19), "f32", t1, 6),
        "turing_19_bf16": (W.turing(shape=SHAPE, stencil=19, sigma=0.3), "bf16", t1, 6),
        "front_19": (W.with_(W.ch_front(shape=SHAPE), stencil=19), "f32", t1, 6),
        "table1_19": (W.with_(W.ch_table1(shape=SHAPE), init="uniform_noise"), "f32", t1, 6),
        "plume_19": (W.with_(W.plume(shape=SHAPE, src=(30, 10, 6)), stencil=19,
                             init="uniform_noise"), "f32", t1, 6),
        "plume_7": (W.with_(W.plume(shape=SHAPE, src=(30, 10, 6)), init="uniform_noise"),
                    "f32", dict(t1, graph=1), 20),
        "resident_diffusion": (W.diffusion_blob(shape=SHAPE), "f32",
                               dict(kernel="resident", plan=(3, 4, 5)), 13),
        "resident_brusselator_periodic": (per_b, "f32",
                                          dict(kernel="resident", plan=(4, 5, 3)), 11),
        "resident_air_bf16": (W.air(SHAPE, src=(9, 4, 3)), "bf16",
                              dict(kernel="resident", plan=(2, 3, 2)), 9),
    }
    return out


def batch_members():
    return [W.ch_front(shape=s, seed=i) for i, s in enumerate([(23, 17, 11), (70, 9, 14),
                                                                (16, 33, 9)])]


def main(path):
    from paper_1004_0480_gb300 import _lib as L
    from paper_1004_0480_gb300.sim import Batch, Sim
    res = {}
    for name, (cfg, storage, tun, steps) in cases().items():
        resident = tun.get("kernel") == "resident"
        with Sim(cfg, storage, tuning=None if resident else tun) as sim:
            if resident:
                sim.set_kernel("resident")
                sim.set_resident_plan(*tun["plan"])
            sim.set_fields(W.initial_fields(cfg))
            sim.step(steps)
            res[f"status_{name}"] = np.array(L.load().rd_sync(sim.ctx))
            res[name] = sim.get_fields()
    cfgs = batch_members()
    sims = [Sim(c) for c in cfgs]
    for c, s in zip(cfgs, sims):
        s.set_fields(W.initial_fields(c))
    b = Batch("ch_front")
    b.set_tuning(tsteps=1, tile_q=16, tile_y=4, zchunk=5, graph=1)
    for s in sims:
        b.add(s)
    b.step(19)
    res["status_batch"] = np.array(L.load().rd_batch_sync(b.b))
    for i, s in enumerate(sims):
        res[f"batch_{i}"] = s.get_fields()
    b.close()
    for s in sims:
        s.close()
    # members advancing their own counts: the CTAs pull their work items
    cfgs = [W.brusselator(shape=s, seed=i) for i, s in enumerate([(23, 17, 11), (70, 9, 14),
                                                                   (16, 33, 9)])]
    sims = [Sim(c) for c in cfgs]
    for c, s in zip(cfgs, sims):
        s.set_fields(W.initial_fields(c))
    b = Batch("brusselator")
    b.set_tuning(tsteps=1, tile_q=16, tile_y=6, zchunk=5, graph=1)
    for s in sims:
        b.add(s)
    b.step_each(dict(zip(sims, [3, 21, 0])))
    res["status_batch_each"] = np.array(L.load().rd_batch_sync(b.b))
    for i, s in enumerate(sims):
        res[f"batch_each_{i}"] = s.get_fields()
    b.close()
    for s in sims:
        s.close()
    np.savez(path, **res)


if __name__ == "__main__":
    main(sys.argv[1])
