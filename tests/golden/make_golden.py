"""Writes ``oracle_regression.json``: FP64 oracle results on small seeded
problems of every family, used to detect any later change of the oracle's
arithmetic.  Calls only ``oracle/`` and the seeded input module.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1004_0480_gb300 import workloads as W  # noqa: E402

CASES = {
    "diffusion_9x8x7": (W.diffusion_blob(shape=(9, 8, 7)), 20),
    "brusselator_periodic_8": (W.brusselator(8), 20),
    "ch_front_10x9x8": (W.ch_front(shape=(10, 9, 8)), 20),
    "air_11x7x6": (W.air((11, 7, 6), src=(4, 3, 2)), 20),
    "brusselator_19pt_neumann_9x8x7": (W.with_(W.brusselator(shape=(9, 8, 7), bc="neumann"),
                                               stencil=19), 20),
    "turing_table1_9x8x7": (W.turing(shape=(9, 8, 7), sigma=0.3), 20),
    "turing_table1_19pt_9x8x7": (W.turing(shape=(9, 8, 7), sigma=0.3, stencil=19), 20),
    "plume_table1_9x8x10": (W.plume(shape=(9, 8, 10), src=(2, 3, 4)), 20),
    "ch_table1_19pt_10x9x8": (W.ch_table1(shape=(10, 9, 8), dt=0.005), 20),
}
SAMPLES = [(0, 0, 0), (1, 2, 3), (5, 4, 2), (6, 6, 5), (3, 0, 1)]   # (x, y, z)


def main():
    out = {}
    for name, (cfg, n) in CASES.items():
        f = W.initial_fields(cfg)
        r = oracle.run(cfg, f, n)
        out[name] = dict(
            steps=n,
            sum=[float(r[s].sum()) for s in range(cfg["nspecies"])],
            sumsq=[float((r[s] ** 2).sum()) for s in range(cfg["nspecies"])],
            samples={f"{x},{y},{z}": [float(r[s, z, y, x]) for s in range(cfg["nspecies"])]
                     for (x, y, z) in SAMPLES})
    with open(os.path.join(HERE, "oracle_regression.json"), "w") as fh:
        json.dump(out, fh, indent=1, sort_keys=True)
        fh.write("\n")


if __name__ == "__main__":
    main()
