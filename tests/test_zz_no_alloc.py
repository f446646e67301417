"""rd_moments_noalloc: the FP64 field moments for callers that cannot
allocate device memory at that point (a thread capturing a CUDA graph, a
serving loop held to a memory budget fixed at start-up, a monitor that must
not trigger the device-wide synchronisation of cudaMalloc / cudaFree).

Through the C ABI, the allocation-free entry point must give the same sums
as rd_mass, the context-based reduction, on two calls in a row.  This file
is named to be collected last, so a run that stops at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_1004_0480_gb300 import workloads as W

pytestmark = pytest.mark.gpu

REL_TOL = 1e-12      # the FP64 reduction tolerance used by the other tests


@pytest.fixture(scope="module")
def rd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1004_0480_gb300 import build as B
    B.build()
    from paper_1004_0480_gb300 import _lib, sim
    return sim, _lib


def field_pointer(sim, storage, level, s):
    """Device address of species s, time level ``level`` of a context whose
    state lives in torch memory (layout documented at rd_attach)."""
    state_bytes, _ = sim_sizes(sim, storage)
    base = (sim._keep[0].data_ptr() + 255) // 256 * 256
    field_bytes = state_bytes // (2 * sim.nspecies)
    return base + (level * sim.nspecies + s) * field_bytes


def sim_sizes(sim, storage):
    from paper_1004_0480_gb300.sim import query_sizes
    return query_sizes(sim.cfg, storage)


def pitch_of(nx, storage):
    per_row = 128 // (2 if storage == "bf16" else 4)
    return (nx + per_row - 1) // per_row * per_row


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_noalloc_moments_match_rd_mass_twice(rd, storage):
    import torch
    simmod, L = rd
    lib = L.load()
    cfg = W.brusselator(shape=(70, 33, 21), seed=7)
    nx, ny, nz = cfg["shape"]
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    with simmod.Sim(cfg, storage, torch_memory=True, tuning=dict(tsteps=1, tile_y=8)) as sim:
        sim.set_fields(W.initial_fields(cfg))
        for rounds in range(2):
            if rounds == 1:
                sim.step(2)          # two launches: level 0 is current again
            for s in range(2):
                ref = sim.mass(s)
                for _ in range(2):   # two calls in a row share the scratch array
                    out.zero_()
                    st = lib.rd_moments_noalloc(
                        ctypes.c_void_p(field_pointer(sim, storage, 0, s)),
                        L.STORAGE[storage], nx, ny, nz, pitch_of(nx, storage),
                        ctypes.c_void_p(out.data_ptr()), None)
                    assert st == L.RD_OK
                    torch.cuda.synchronize()
                    got = out.cpu().numpy()
                    assert got[2] == ref[2] == 0
                    np.testing.assert_allclose(got[:2], ref[:2], rtol=REL_TOL, atol=0)


def test_noalloc_rejects_bad_sizes(rd):
    import torch
    _, L = rd
    lib = L.load()
    buf = torch.zeros(64, dtype=torch.float32, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    p, o = ctypes.c_void_p(buf.data_ptr()), ctypes.c_void_p(out.data_ptr())
    assert lib.rd_moments_noalloc(p, 0, 0, 1, 1, 1, o, None) == L.RD_EINVAL
    assert lib.rd_moments_noalloc(p, 0, 8, 1, 1, 4, o, None) == L.RD_EINVAL
    assert lib.rd_moments_noalloc(p, 0, 8, 2 ** 16, 2 ** 16, 8, o, None) == L.RD_EINVAL
    assert lib.rd_moments_noalloc(p, 7, 8, 1, 1, 8, o, None) == L.RD_EINVAL
    assert lib.rd_moments_noalloc(None, 0, 8, 1, 1, 8, o, None) == L.RD_EINVAL


def test_noalloc_counts_nonfinite_on_a_stream(rd):
    """A NaN and an Inf in the field: the count is 2 and the sums run over
    the finite cells only, as rd_mass gives; the call runs on a caller's
    stream (its handle passed through the ABI), twice in a row."""
    import torch
    simmod, L = rd
    lib = L.load()
    cfg = W.diffusion_blob(shape=(45, 19, 13), seed=3)
    nx, ny, nz = cfg["shape"]
    f = W.initial_fields(cfg)
    f[0, 4, 7, 11] = np.nan
    f[0, 12, 18, 44] = np.inf
    finite = f[0][np.isfinite(f[0])].astype(np.float64)
    stream = torch.cuda.Stream()
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    with simmod.Sim(cfg, "f32", torch_memory=True) as sim:
        sim.set_fields(f)
        ref = sim.mass(0)
        assert ref[2] == 2
        torch.cuda.synchronize()
        for _ in range(2):
            with torch.cuda.stream(stream):
                out.zero_()
            st = lib.rd_moments_noalloc(
                ctypes.c_void_p(field_pointer(sim, "f32", 0, 0)), L.STORAGE["f32"], nx, ny, nz,
                pitch_of(nx, "f32"), ctypes.c_void_p(out.data_ptr()),
                ctypes.c_void_p(stream.cuda_stream))
            assert st == L.RD_OK
            stream.synchronize()
            got = out.cpu().numpy()
            assert got[2] == 2
            np.testing.assert_allclose(got[:2], ref[:2], rtol=REL_TOL, atol=0)
            np.testing.assert_allclose(got[0], finite.sum(), rtol=1e-12)
            np.testing.assert_allclose(got[1], (finite ** 2).sum(), rtol=1e-12)
