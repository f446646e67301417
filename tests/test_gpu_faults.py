"""Failure paths, made on the host: allocation failures injected with
rd_debug_fail_alloc (the k-th device or pinned-host allocation fails as if
memory were exhausted).  Each must return RD_ENOMEM, free what the call had
obtained (the device's free memory returns to where it was), and leave the
library usable.  No GPU fault is involved."""
import ctypes

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
    from paper_1004_0480_gb300 import _lib, sim
    return sim, _lib


def free_bytes():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_context_creation_survives_each_failed_allocation(rd):
    sim, L = rd
    lib = L.load()
    # large enough that a leaked state or scratch buffer shows in the free memory
    cfg = W.brusselator(shape=(256, 256, 64))
    conf = sim.make_config(cfg)
    with sim.Sim(cfg):
        pass                                  # first use: module loading
    base = free_bytes()
    for k in (1, 2):                          # the state, then the scratch
        assert lib.rd_debug_fail_alloc(k) == L.RD_OK
        ctx = ctypes.c_void_p()
        assert lib.rd_create(ctypes.byref(conf), ctypes.byref(ctx)) == L.RD_ENOMEM
        assert not ctx.value
        assert b"cudaMalloc" in lib.rd_last_error(None)
        assert abs(free_bytes() - base) < (1 << 20), f"allocation {k}: memory leaked"
    lib.rd_debug_fail_alloc(0)
    # the library still works: a context steps and matches a fresh run
    f = W.initial_fields(cfg)
    with sim.Sim(cfg) as s:
        s.set_fields(f)
        s.step(3)
        a = s.get_fields()
    with sim.Sim(cfg) as s:
        s.set_fields(f)
        s.step(3)
        assert np.array_equal(a, s.get_fields())
    assert abs(free_bytes() - base) < (1 << 20)
    assert lib.rd_debug_fail_alloc(-1) == L.RD_EINVAL


def test_batch_descriptor_allocation_failure(rd):
    sim, L = rd
    lib = L.load()
    cfgs = [W.brusselator(shape=(40, 24, 20), seed=i) for i in range(3)]
    sims = [sim.Sim(c) for c in cfgs]
    ref = []
    for c in cfgs:
        with sim.Sim(c) as s:
            s.set_fields(W.initial_fields(c))
            s.step(5)
            ref.append(s.get_fields())
    try:
        for c, s in zip(cfgs, sims):
            s.set_fields(W.initial_fields(c))
        b = sim.Batch("brusselator")
        for s in sims:
            b.add(s)
        for k in (1, 2):                      # the device array, then the pinned one
            lib.rd_debug_fail_alloc(k)
            assert lib.rd_batch_step(b.b, 5) == L.RD_ENOMEM
        lib.rd_debug_fail_alloc(0)
        # nothing was stepped by the failed calls; the batch works afterwards
        b.step(5)
        b.sync()
        for s, r in zip(sims, ref):
            assert np.array_equal(s.get_fields(), r)
        b.close()
    finally:
        lib.rd_debug_fail_alloc(0)
        for s in sims:
            s.close()
