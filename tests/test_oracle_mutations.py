"""Planted mistakes in the oracle must fail at least one pin (CPU only).

Each case compiles a copy of oracle/ptrig_oracle.c with one plausible mistake
(a wrong coefficient, sign, index, constant or dropped term), loads it as a
separate oracle instance and runs the pin suite against it.
"""
import importlib.util
import os
import subprocess
import tempfile

import pytest

import tests.test_oracle_pins as pins

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "ptrig_oracle.c")

MUTATIONS = {
    "coefficient_C5": ("static const int QC[6] = {-1, -4, -5, -13, -10, -11};",
                       "static const int QC[6] = {-1, -4, -5, -13, -10, -10};"),
    "coefficient_B3": ("static const int QB[6] = {0, 10, 46, 217, 297, 542};",
                       "static const int QB[6] = {0, 10, 46, 216, 297, 542};"),
    "denominator_sign": ("  double D = c * u + d;\n  if (func == 2) return N / D;",
                         "  double D = c * u - d;\n  if (func == 2) return N / D;"),
    "sin_cos_swapped": ("return (func == 0) ? N / h : D / h;", "return (func == 0) ? D / h : N / h;"),
    "quadrant_sign": ("s = (r->q == 0 || r->q == 1) ? 1.0 : -1.0;", "s = (r->q == 0 || r->q == 2) ? 1.0 : -1.0;"),
    "cos_made_odd": ("    s = (r->q == 0 || r->q == 3) ? 1.0 : -1.0;\n",
                     "    s = (r->q == 0 || r->q == 3) ? 1.0 : -1.0;\n    if (r->neg) s = -s;\n"),
    "no_complement": ("  if (q & 1) {\n    /* F <- 2^S - F", "  if (0) {\n    /* F <- 2^S - F"),
    "window_off_by_one": ("int i0 = (e >= 2) ? (e - 2) / 32 : 0;", "int i0 = (e >= 2) ? (e - 2) / 32 + 1 : 0;"),
    "degree_factor": ("double R = 180.0 / g_pi;", "double R = 180.0 / 3.1416;"),
    "segment_width": ("int k = (int)floor(u / (g_pi / 12.0));", "int k = (int)floor(u / 0.261);"),
    "taylor_no_alternation": ("s += ((i % 2) ? -1.0 : 1.0) * pow(u, 2 * i + 1) / fact;",
                              "s += pow(u, 2 * i + 1) / fact;"),
    "taylor_tan_coefficient": ("static const double TAN_NUM[9] = {1.0, 1.0, 2.0, 17.0,",
                               "static const double TAN_NUM[9] = {1.0, 1.0, 2.0, 16.0,"),
    "derivative_chain_sign": ("double du_dx = ((r.q % 2) ? -1.0 : 1.0) * (r.neg ? -1.0 : 1.0);",
                              "double du_dx = (r.neg ? -1.0 : 1.0);"),
    "derivative_delta": ("double Delta = a * d - b * c;", "double Delta = a * d + b * c;"),
    "fisr_magic": ("i = 0x5fe6eb50c7b537a9ull - (i >> 1);", "i = 0x5fe6eb50c7b537a9ull - (i >> 2);"),
    "faithful_selector": ("int k = (int)floor(u / 0.261);\n  if (k > 5) k = 5;",
                          "int k = (int)floor(u / 0.2618);\n  if (k > 5) k = 5;"),
    "faithful_newton": ("y = y * (1.5 - (v * 0.5) * y * y);", "y = y * (1.5 - (v * 0.25) * y * y);"),
    "neighbour_direction": ("  int k = segment(r.u) + dk;\n", "  int k = segment(r.u) - dk;\n"),
    "neighbour_ignores_shift": ("  int k = segment(r.u) + dk;\n", "  int k = segment(r.u) + 0 * dk;\n"),
    "neighbour_clamp": ("  int k = segment(r.u) + dk;\n  if (k < 0) k = 0;", "  int k = segment(r.u) + dk;\n  if (k < 0) k = 1;"),
}

PIN_TESTS = [getattr(pins, n) for n in dir(pins) if n.startswith("test_")]


def _load_mutant(name, src_text, tmpdir):
    c_path = os.path.join(tmpdir, f"mut_{name}.c")
    so_path = os.path.join(tmpdir, f"libmut_{name}.so")
    with open(c_path, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off", c_path,
                    "-o", so_path, "-lm"], check=True)
    spec = importlib.util.spec_from_file_location(f"oracle_mutant_{name}",
                                                  os.path.join(ROOT, "oracle", "ptrig_oracle.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod._SRC = c_path
    mod._LIB = so_path
    mod.lib()
    return mod


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    with tempfile.TemporaryDirectory() as td:
        mod = _load_mutant(name, src.replace(old, new), td)
        failed = []
        for t in PIN_TESTS:
            try:
                t(mod) if t.__code__.co_argcount == 1 else t()
            except (AssertionError, ValueError, ZeroDivisionError):
                failed.append(t.__name__)
            except pytest.skip.Exception:
                pass
        assert failed, f"no pin caught the planted mistake {name}"
