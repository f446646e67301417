"""The C ABI library loads on a machine without a GPU, exports every function
``include/rd.h`` declares, and the ctypes binding agrees with the C layout.
Only host-side validation is called here (no device work)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1004_0480_gb300 import _lib as L
from paper_1004_0480_gb300 import build as B
from paper_1004_0480_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rd.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rd_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 25
    for n in names:
        assert hasattr(lib, n), f"{n} declared in rd.h but not exported"
    assert set(names) == set(L.SIGNATURES), "ctypes table out of sync with rd.h"


def test_struct_layout_matches_c(tmp_path):
    probe = tmp_path / "probe.c"
    probe.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "rd.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(rd_config),
         offsetof(rd_config, D), offsetof(rd_config, bc), offsetof(rd_config, bc_value),
         offsetof(rd_config, params), offsetof(rd_config, wind_u0), offsetof(rd_config, src_rate),
         sizeof(rd_tuning), offsetof(rd_config, stencil), offsetof(rd_config, wind_vel),
         offsetof(rd_config, wind_tau));
  return 0;
}''')
    exe = tmp_path / "probe"
    subprocess.run(["gcc", f"-I{os.path.join(ROOT, 'include')}", str(probe), "-o", str(exe)],
                   check=True)
    vals = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True,
                                        check=True).stdout.split()))
    C = L.RdConfig
    assert vals == [ctypes.sizeof(C), C.D.offset, C.bc.offset, C.bc_value.offset,
                    C.params.offset, C.wind_u0.offset, C.src_rate.offset,
                    ctypes.sizeof(L.RdTuning), C.stencil.offset, C.wind_vel.offset,
                    C.wind_tau.offset]


def test_binding_constants_match_the_header_enums():
    text = open(HEADER).read()
    enum = {m.group(1): int(m.group(2))
            for m in re.finditer(r"\b(RD_[A-Z0-9_]+)\s*=\s*(\d+)", text)}
    prefixed = {"RD_BC_": L.BC, "RD_MODEL_": L.MODEL, "RD_STORE_": L.STORAGE,
                "RD_WIND_": L.WIND, "RD_KERNEL_": L.KERNEL}
    for prefix, table in prefixed.items():
        in_header = {k for k in enum if k.startswith(prefix)}
        named = {prefix + ("none" if k is None else k).upper(): v for k, v in table.items()}
        assert set(named) == in_header, prefix
        for name, value in named.items():
            assert enum[name] == value, name
    assert [enum[k] for k in ("RD_OK", "RD_EINVAL", "RD_EUNSTABLE", "RD_EUNSUPPORTED")] == \
        [L.RD_OK, L.RD_EINVAL, L.RD_EUNSTABLE, L.RD_EUNSUPPORTED]
    assert (enum["RD_FLAG_NO_ALLOC"], enum["RD_FLAG_FORCE"]) == (L.FLAG_NO_ALLOC, L.FLAG_FORCE)


def test_status_strings(lib):
    for st in range(9):
        assert lib.rd_status_str(st)
    assert lib.rd_status_str(99) == b"unknown status"


def _cfg(cfg, **kw):
    from paper_1004_0480_gb300.sim import make_config
    c = make_config(cfg)
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def test_validation_host_only(lib):
    sz = ctypes.c_size_t()
    sc = ctypes.c_size_t()
    q = lambda c: lib.rd_query_sizes(ctypes.byref(c), ctypes.byref(sz), ctypes.byref(sc))
    assert q(_cfg(W.cfg_brusselator_256())) == L.RD_OK
    # two levels of two species, rows padded to 128 bytes
    assert sz.value == 2 * 2 * 256 * 256 * 256 * 4
    # stability: dt <= h^2 / (6 D) for isotropic diffusion
    ok = W.diffusion_blob(8, dt=1.0 / 6.0)
    bad = W.diffusion_blob(8, dt=1.0 / 6.0 * 1.001)
    assert q(_cfg(ok)) == L.RD_OK
    assert q(_cfg(bad)) == L.RD_EUNSTABLE
    c = _cfg(bad)
    c.flags = L.FLAG_FORCE
    assert q(c) == L.RD_OK
    # the air problem's Courant number enters the bound
    air = W.air((16, 16, 8), src=(1, 1, 1), dt=0.2)
    assert q(_cfg(air)) == L.RD_OK
    assert q(_cfg(W.with_(air, dt=0.8))) == L.RD_EUNSTABLE
    # grid and species checks
    assert q(_cfg(W.diffusion_blob(8), nx=1)) == L.RD_EINVAL
    assert q(_cfg(W.brusselator(8), nspecies=3)) == L.RD_EINVAL
    c = _cfg(W.brusselator(8))
    c.bc[0][0] = L.BC["neumann"]          # unpaired periodic face
    assert q(c) == L.RD_EINVAL
    c = _cfg(W.ch_front(8))
    c.bc[2][4] = L.BC["dirichlet"]        # no held layer on the CH species
    assert q(c) == L.RD_EUNSUPPORTED
    c = _cfg(W.ch_front(8))
    c.wind_kind, c.wind_u0 = 1, 0.5       # the front model has no wind
    assert q(c) == L.RD_EUNSUPPORTED
    c = _cfg(W.ch_front(8))
    c.src_species, c.src_x, c.src_y, c.src_z = 2, 1, 1, 1   # nor a source on c
    assert q(c) == L.RD_EUNSUPPORTED
    c.src_species = 0                     # a source on a is fine
    assert q(c) == L.RD_OK
    c = _cfg(W.air((8, 8, 8), src=(1, 1, 1)))
    c.wind_u0 = float("nan")              # wind speed must be finite
    assert q(c) == L.RD_EINVAL
    c = _cfg(W.air((8, 8, 8), src=(1, 1, 1)))
    c.src_x = 8                           # source outside the grid
    assert q(c) == L.RD_EINVAL
    assert b"source" in lib.rd_last_error(None)


def test_validation_of_the_19_point_stencil(lib):
    sz = ctypes.c_size_t()
    q = lambda c: lib.rd_query_sizes(ctypes.byref(c), ctypes.byref(sz), None)
    b19 = W.with_(W.brusselator(8), stencil=19)
    assert q(_cfg(b19)) == L.RD_OK
    assert q(_cfg(b19, stencil=0)) == L.RD_OK       # 0 means the 7-point default
    assert q(_cfg(b19, stencil=13)) == L.RD_EINVAL
    # one diffusivity per species
    c = _cfg(b19)
    c.D[1][2] = 1.0
    assert q(c) == L.RD_EINVAL
    assert b"diffusivity" in lib.rd_last_error(None)
    # the Cahn-Hilliard models take the 19-point stencil too; their scratch
    # then holds one more float field, mu (rows of 8 cells padded to 32)
    xb7, xb19 = ctypes.c_size_t(), ctypes.c_size_t()
    for model in (W.ch_front(8), W.ch_table1(shape=(8, 8, 8))):
        assert lib.rd_query_sizes(ctypes.byref(_cfg(W.with_(model, stencil=19))), None,
                                  ctypes.byref(xb19)) == L.RD_OK
        assert lib.rd_query_sizes(ctypes.byref(_cfg(W.with_(model, stencil=7, dt=0.005))),
                                  None, ctypes.byref(xb7)) == L.RD_OK
        assert xb19.value - xb7.value == 8 * 8 * 32 * 4
    # stability: the update's centre weight is 1 - 4 D dt / h^2 (19-point)
    # against 1 - 6 D dt / h^2 (7-point)
    ok = W.with_(W.diffusion_blob(8, dt=0.25), stencil=19)
    bad = W.with_(W.diffusion_blob(8, dt=0.25 * 1.001), stencil=19)
    assert q(_cfg(ok)) == L.RD_OK
    assert q(_cfg(bad)) == L.RD_EUNSTABLE
    assert q(_cfg(W.with_(ok, stencil=7))) == L.RD_EUNSTABLE
    # an isotropic air problem with wind and a source is accepted
    air = W.with_(W.air((16, 16, 8), src=(1, 1, 1), dt=0.2), stencil=19, D=[[0.1] * 3] * 3)
    assert q(_cfg(air)) == L.RD_OK


def test_validation_of_the_turing_model(lib):
    sz = ctypes.c_size_t()
    q = lambda c: lib.rd_query_sizes(ctypes.byref(c), ctypes.byref(sz), None)
    cfg = W.turing(shape=(16, 8, 8))
    assert q(_cfg(cfg)) == L.RD_OK
    assert sz.value == 2 * 2 * 8 * 8 * 32 * 4      # rows of 16 cells padded to 32
    assert q(_cfg(cfg, nspecies=3)) == L.RD_EINVAL
    assert q(_cfg(W.with_(cfg, stencil=19))) == L.RD_OK
    # the Table 1 time step is inside both stencils' bounds; ten times it is not
    assert q(_cfg(W.with_(cfg, dt=cfg["dt"] * 10))) == L.RD_EUNSTABLE
    assert q(_cfg(cfg, model=6)) == L.RD_EINVAL


def test_bf16_rows_are_128_bytes(lib):
    from paper_1004_0480_gb300.sim import make_config
    c = make_config(W.diffusion_blob(shape=(70, 3, 2)), storage="bf16")
    sz = ctypes.c_size_t()
    assert lib.rd_query_sizes(ctypes.byref(c), ctypes.byref(sz), None) == L.RD_OK
    # 70 cells pad to 128 bf16 per row: 2 levels * 1 species * 128*3*2 * 2 bytes
    assert sz.value == 2 * ((128 * 3 * 2 * 2 + 255) // 256 * 256)


def test_validation_of_the_table1_cahn_hilliard_model(lib):
    sz = ctypes.c_size_t()
    q = lambda c: lib.rd_query_sizes(ctypes.byref(c), ctypes.byref(sz), None)
    cfg = W.ch_table1(shape=(16, 8, 8))          # the paper's dt = 0.02, 19-point
    assert q(_cfg(cfg)) == L.RD_OK
    # dt lambda L (sigma L + 3 gamma - eps) <= 2: 0.78 with L = 16/3 (19-point),
    # 3.36 with L = 12 (7-point), which needs dt <= 2 / 168
    assert q(_cfg(W.with_(cfg, stencil=7))) == L.RD_EUNSTABLE
    assert q(_cfg(W.with_(cfg, stencil=7, dt=2.0 / 168))) == L.RD_OK
    assert q(_cfg(W.with_(cfg, stencil=7, dt=2.0 / 168 * 1.001))) == L.RD_EUNSTABLE
    assert q(_cfg(cfg, nspecies=2)) == L.RD_EINVAL
    c = _cfg(cfg)
    c.D[2][0] = c.D[2][1] = c.D[2][2] = 0.5      # c3 has no Fickian term
    assert q(c) == L.RD_EUNSUPPORTED
    c = _cfg(cfg)
    c.bc[2][0] = L.BC["dirichlet"]               # no held layer on c3
    assert q(c) == L.RD_EUNSUPPORTED


def test_batch_step_counts_are_in_member_order_and_name_only_members():
    from paper_1004_0480_gb300.sim import member_counts

    class M:   # stands in for a Sim (members are compared by identity)
        pass

    a, b, c, stranger = M(), M(), M(), M()
    assert member_counts([a, b, c], {c: 7, a: 2}) == [2, 0, 7]
    assert member_counts([], {}) == []
    with pytest.raises(ValueError):
        member_counts([a, b], {a: 1, stranger: 3})
