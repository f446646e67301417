"""The bounds-checked debug build (RD_BOUNDS_CHECK=1, rd_debug_bounds): a
stand-in for a memory checker.  Every step-kernel family runs small problems
under it; no out-of-range access may be recorded, and the results must equal
the normal library's bit for bit (the checks only skip accesses that are out
of range).  The recording path itself is exercised by the self-test, which
records a violation without touching memory.  Nothing here faults the GPU:
an out-of-range access is never made, only recorded."""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1004_0480_gb300 import build as B
    B.build()
    return B


def run_cases(tmp_path, debug):
    out = tmp_path / ("debug.npz" if debug else "normal.npz")
    env = dict(os.environ, RD_BOUNDS_CHECK="1" if debug else "0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "bounds_cases.py"), str(out)],
                       env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    return dict(np.load(out))


def test_every_kernel_family_runs_clean_under_the_bounds_checks(built, tmp_path):
    dbg = run_cases(tmp_path, True)
    ref = run_cases(tmp_path, False)
    assert set(dbg) == set(ref)
    for k in sorted(dbg):
        if k.startswith("status_"):
            assert int(dbg[k]) == 0 and int(ref[k]) == 0, f"{k}: {int(dbg[k])}"
        else:
            assert np.array_equal(dbg[k].view(np.uint32), ref[k].view(np.uint32)), k


SELFTEST = r"""
import ctypes, os, sys
sys.path.insert(0, {root!r})
from paper_1004_0480_gb300 import _lib as L
lib = L.load()
w = ctypes.c_uint64()
assert lib.rd_debug_bounds(ctypes.byref(w), 2) == L.RD_OK
assert w.value >> 63 == 1 and (w.value >> 40) & 0xFFFF == 0xFFFF, hex(w.value)
assert lib.rd_debug_bounds(ctypes.byref(w), 0) == L.RD_OK and w.value == 0
print("ok")
"""


def test_the_debug_build_records_without_touching_memory(built):
    env = dict(os.environ, RD_BOUNDS_CHECK="1")
    r = subprocess.run([sys.executable, "-c", SELFTEST.format(root=ROOT)], env=env,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "ok" in r.stdout, r.stderr[-3000:]
    # the normal build has no checks
    from paper_1004_0480_gb300 import _lib as L
    w = ctypes.c_uint64()
    assert L.load().rd_debug_bounds(ctypes.byref(w), 0) == L.RD_EUNSUPPORTED
