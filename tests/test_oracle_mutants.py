"""The oracle's pins must catch plausible mistakes.

Each mutant below is a one-token slip planted in a temporary copy of the C
oracle (compiled on the CPU into a temp directory; the committed oracle is
never touched).  The closed-form and invariant pins of
``test_oracle_pins.py`` -- not the NumPy cross-check -- are run against
the mutant, and at least one of them must fail.
"""
import ctypes
import inspect
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "rd_oracle.c")

MUTANTS = {
    "neumann_ghost_off_by_one": ("return n - 1;", "return n - 2;"),
    "periodic_wrap_off_by_one": ("return i + n;", "return i + n - 1;"),
    "laplacian_centre_weight": ("(m + q - 2.0 * c)", "(m + q - 2.5 * c)"),
    "diffusivity_axes_swapped": ("p->D[s][a] * second_diff", "p->D[s][2 - a] * second_diff"),
    "upwind_wrong_side": ("rate -= u * (v[s] - nb(p, f, s, x, y, z, 0, -1)) / p->h;",
                          "rate -= u * (nb(p, f, s, x, y, z, 0, +1) - v[s]) / p->h;"),
    "wind_height_index": ("log(1.0 + (double)z)", "log(2.0 + (double)z)"),
    "brusselator_cubic_term": ("r[1] = b * u - u * u * w;", "r[1] = b * u - u * w * w;"),
    "brusselator_linear_term": ("(b + 1.0) * u", "b * u"),
    "ch_kappa_sign": ("fp - kappa * laplacian", "fp + kappa * laplacian"),
    "ch_double_well": ("2.0 * cc * (cc - 1.0) * (2.0 * cc - 1.0)", "2.0 * cc * (cc - 1.0)"),
    "ch_mobility_dropped": ("rate += p->p[1] * laplacian(p, mu, 2, x, y, z);",
                            "rate += laplacian(p, mu, 2, x, y, z);"),
    "air_ozone_sign": ("r[2] = ph - ti;", "r[2] = ti - ph;"),
    "air_titration_species": ("double ti = k * v[0] * v[2];", "double ti = k * v[0] * v[1];"),
    "source_x_y_swapped": ("x == p->src_x && y == p->src_y", "x == p->src_y && y == p->src_x"),
    "held_layer_inset": ("int at = (f % 2 == 0) ? 0 : ext[axis] - 1;",
                         "int at = (f % 2 == 0) ? 1 : ext[axis] - 1;"),
    "front_reaction_sign": ("r[2] = q;", "r[2] = -q;"),
    "euler_half_step": ("double out = v[s] + p->dt * rate;",
                        "double out = v[s] + 0.5 * p->dt * rate;"),
    "turing_cubic_term": ("r[0] = c1 - c1 * c1 * c1 - c2;", "r[0] = c1 - c1 * c1 - c2;"),
    "turing_alpha_dropped": ("(c1 - alpha * c2 - beta)", "(c1 - c2 - beta)"),
    "turing_gamma_dropped": ("r[1] = gamma * (", "r[1] = ("),
    "wind3_time_of_step": ("wind3(p, (double)n * p->dt, u3)", "wind3(p, (double)(n + 1) * p->dt, u3)"),
    "wind3_uz_phase": ("u[2] = p->w3[2] * sin(t / p->w3[3]);", "u[2] = p->w3[2] * cos(t / p->w3[3]);"),
    "wind3_uy_from_ux": ("u[1] = p->w3[1];", "u[1] = p->w3[0];"),
    "upwind_forward_difference": ("if (u < 0.0) return -u * (nb(p, f, s, x, y, z, axis, +1) - c) / p->h;",
                                  "if (u < 0.0) return -u * (c - nb(p, f, s, x, y, z, axis, -1)) / p->h;"),
    "ch1_sink_sign": ("r[0] = -k1 * c1 * c2 - k2 * c1 * c3;", "r[0] = -k1 * c1 * c2 + k2 * c1 * c3;"),
    "ch1_sink_missing_in_c3": ("r[2] = k1 * c1 * c2 - k2 * c1 * c3;", "r[2] = k1 * c1 * c2;"),
    "ch1_sigma_sign": ("+ sigma * laplacian(p, c, 2, x, y, z);", "- sigma * laplacian(p, c, 2, x, y, z);"),
    "ch1_lambda_sign": ("rate -= p->p[2] * laplacian(p, mu, 2, x, y, z);",
                        "rate += p->p[2] * laplacian(p, mu, 2, x, y, z);"),
    "ch1_cubic_power": ("gamma * cc * cc * cc", "gamma * cc * cc"),
    "stencil19_centre_weight": ("{{1, 2, 1}, {2, -24, 2}, {1, 2, 1}}",
                                "{{1, 2, 1}, {2, -26, 2}, {1, 2, 1}}"),
    "stencil19_diagonals_doubled": ("{{1, 2, 1}, {2, -24, 2}, {1, 2, 1}}",
                                    "{{2, 2, 2}, {2, -28, 2}, {2, 2, 2}}"),
    "stencil19_corners_for_edges": ("/* r = -1 */ {{0, 1, 0}, {1, 2, 1}, {0, 1, 0}}",
                                    "/* r = -1 */ {{1, 0, 1}, {0, 2, 0}, {1, 0, 1}}"),
    "stencil19_normalisation": ("acc / (6.0 * p->h * p->h)", "acc / (4.0 * p->h * p->h)"),
    "stencil19_edge_ghost_rule": ("int Y = ghost_index(y + dy, p->ny, p->bc[s][2], p->bc[s][3]);",
                                  "int Y = ghost_index(y + dy, p->ny, p->bc[s][0], p->bc[s][1]);"),
}

# pins that stand on their own (the NumPy cross-check is excluded)
PIN_FUNCS = [f for name, f in inspect.getmembers(pins, inspect.isfunction)
             if name.startswith("test_") and name != "test_oracles_agree_on_every_family"]


class _Shim:
    """Looks like the ``oracle`` package but runs a mutant library."""

    def __init__(self, lib):
        self._lib = lib
        self.np_run = oracle.np_run

    def run(self, cfg, fields, nsteps, n0=0):
        nx, ny, nz = cfg["shape"]
        st = np.ascontiguousarray(np.asarray(fields, dtype=np.float64)).copy()
        p = oracle.make_problem(cfg)
        p.n0 = int(n0)
        rc = self._lib.orc_run(ctypes.byref(p),
                               st.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                               int(nsteps))
        if rc != 0:
            raise ValueError("rejected")
        return st


def _param_sets(func):
    marks = getattr(func, "pytestmark", [])
    sets = [{}]
    for m in marks:
        if m.name != "parametrize":
            continue
        names = [n.strip() for n in m.args[0].split(",")]
        new = []
        for s in sets:
            for v in m.args[1]:
                vals = v if len(names) > 1 else (v,)
                d = dict(s)
                d.update(zip(names, vals))
                new.append(d)
        sets = new
    return sets


def _pins_fail(shim):
    failed = []
    for f in PIN_FUNCS:
        for kw in _param_sets(f):
            if kw.get("impl") == "np":
                continue
            try:
                f(shim, **kw)
            except Exception:  # noqa: BLE001 -- any failure counts
                failed.append(f.__name__)
    return failed


def test_pin_set_is_green_on_the_committed_oracle(orc):
    assert _pins_fail(_Shim(orc._load())) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not unique: {old!r}"
    msrc = tmp_path / "mut.c"
    msrc.write_text(src.replace(old, new))
    hdr_dir = os.path.dirname(SRC)
    so = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                    f"-I{hdr_dir}", str(msrc), "-o", str(so), "-lm"], check=True)
    lib = ctypes.CDLL(str(so))
    lib.orc_run.argtypes = [ctypes.POINTER(oracle.OrcProblem),
                            ctypes.POINTER(ctypes.c_double), ctypes.c_int64]
    lib.orc_run.restype = ctypes.c_int
    assert _pins_fail(_Shim(lib)), f"mutant {name} survived every pin"
