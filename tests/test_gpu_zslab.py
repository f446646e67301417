"""The device path of the z-slab decomposition on one GPU: the slabs of 2
and 3 ranks held by one process (``DeviceSlab``: fields resident on the GPU,
ghost planes moved with rd_copy_planes, steps with rd_step), exchanged by
``exchange_local`` -- the messages of ``exchange`` without a collective, so
no kernel waits on another.  Owned planes must equal the undivided run bit
for bit (every owned cell has the neighbours and arithmetic of the undivided
grid), and the owned-plane FP64 moments must add up to rd_mass of the
undivided field.  The NCCL transport between GPUs is not run here (one GPU
per run)."""
import ctypes

import numpy as np
import pytest

from paper_1004_0480_gb300 import workloads as W
from paper_1004_0480_gb300 import zslab as Z

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


def cases():
    air = W.air((40, 18, 24), src=(7, 9, 13))
    air["wind"] = dict(kind="const", u0=0.7)
    air["bc"][0][5] = "dirichlet"
    air["bc_value"] = [[0.0] * 5 + [0.05], [0.0] * 6, [0.0] * 6]
    plume = W.with_(W.plume(shape=(40, 30, 36), src=(10, 15, 20)), init="uniform_noise")
    return {
        "brusselator_periodic": (W.brusselator(shape=(70, 20, 26)), "f32"),
        "brusselator_periodic_bf16": (W.brusselator(shape=(70, 20, 26)), "bf16"),
        "front_halo2_held": (W.ch_front(shape=(40, 20, 30)), "f32"),
        "air_wind_held_top": (air, "f32"),
        "turing_19pt": (W.turing(shape=(48, 20, 27), stencil=19, sigma=0.3), "f32"),
        "table1_19pt_ch": (W.with_(W.ch_table1(shape=(36, 20, 30)), init="uniform_noise"), "f32"),
        "plume_3d_wind": (plume, "f32"),
    }


CASES = cases()
STEPS = 23


@pytest.mark.parametrize("ws", [2, 3])
@pytest.mark.parametrize("name", sorted(CASES))
def test_device_slabs_equal_the_undivided_grid(rd, name, ws):
    import torch
    sim, _ = rd
    cfg, storage = CASES[name]
    f = W.initial_fields(cfg)
    with sim.Sim(cfg, storage, stream=torch.cuda.current_stream()) as whole:
        whole.set_fields(f)
        whole.step(STEPS)
        ref = whole.get_fields()
        ref_mass = [whole.mass(s) for s in range(cfg["nspecies"])]
    plans = [Z.plan(cfg, ws, r) for r in range(ws)]
    slabs = [Z.DeviceSlab(p, storage) for p in plans]
    try:
        for slab, p in zip(slabs, plans):
            slab.set_fields(Z.scatter(f, p))
        Z.run_local(slabs, plans, STEPS)
        got = np.empty_like(ref)
        for slab, p in zip(slabs, plans):
            got[:, p.z0:p.z1] = slab.owned_fields()
        assert np.array_equal(got.view(np.uint32), ref.view(np.uint32)), name
        for s in range(cfg["nspecies"]):
            tot = sum(slab.moments(s).cpu().numpy() for slab in slabs)
            np.testing.assert_allclose(tot[:2], ref_mass[s][:2], rtol=1e-12)
            assert tot[2] == ref_mass[s][2] == 0
    finally:
        for slab in slabs:
            slab.close()


def test_copy_planes_round_trip_and_refusals(rd):
    import torch
    sim, L = rd
    cfg = W.air((37, 11, 9), src=(3, 4, 5))
    f = W.initial_fields(cfg)
    with sim.Sim(cfg) as s:
        s.set_fields(f)
        pb = s.plane_bytes
        assert pb == 11 * 64 * 4                # rows of 37 cells padded to 64
        buf = torch.empty(3 * pb, dtype=torch.uint8, device="cuda")
        s.copy_planes(1, 4, 3, buf, to_buf=True)
        planes = buf.view(torch.float32).view(3, 11, 64)[:, :, :37].cpu().numpy()
        assert np.array_equal(planes, f[1, 4:7])
        doubled = (buf.view(torch.float32) * 2).view(torch.uint8).contiguous()
        s.copy_planes(1, 4, 3, doubled, to_buf=False)
        s.sync()
        g = s.get_field(1)
        assert np.array_equal(g[4:7], 2 * f[1, 4:7]) and np.array_equal(g[:4], f[1, :4])
        lib = L.load()
        bad = [(1, 7, 3, buf.data_ptr(), 3 * pb),       # planes beyond the grid
               (1, 0, 3, buf.data_ptr(), 3 * pb - 4),   # wrong size
               (3, 0, 3, buf.data_ptr(), 3 * pb)]       # no such species
        for sp, z0, k, ptr, nb in bad:
            assert lib.rd_copy_planes(s.ctx, sp, z0, k, ctypes.c_void_p(ptr), nb, 1) == L.RD_EINVAL
        host = np.zeros(3 * pb, dtype=np.uint8)
        assert lib.rd_copy_planes(s.ctx, 0, 0, 3, ctypes.c_void_p(host.ctypes.data), 3 * pb,
                                  1) == L.RD_EINVAL
