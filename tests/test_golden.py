"""The oracle reproduces its committed regression fixture exactly (up to
summation rounding), so any change to its arithmetic is visible."""
import json
import os

import numpy as np

from paper_1004_0480_gb300 import workloads as W

HERE = os.path.join(os.path.dirname(__file__), "golden")


def test_oracle_matches_regression_fixture(orc):
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    ref = json.load(open(os.path.join(HERE, "oracle_regression.json")))
    assert set(ref) == set(mg.CASES)
    for name, (cfg, n) in mg.CASES.items():
        r = orc.run(cfg, W.initial_fields(cfg), ref[name]["steps"])
        for s in range(cfg["nspecies"]):
            assert abs(r[s].sum() - ref[name]["sum"][s]) <= 1e-12 * max(1.0, abs(ref[name]["sum"][s]))
            assert abs((r[s] ** 2).sum() - ref[name]["sumsq"][s]) <= 1e-12 * max(1.0, ref[name]["sumsq"][s])
        for key, vals in ref[name]["samples"].items():
            x, y, z = map(int, key.split(","))
            np.testing.assert_allclose(r[:, z, y, x], np.array(vals), rtol=1e-13, atol=0)
