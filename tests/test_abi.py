"""CPU checks of the C ABI library: it builds for sm_103a, loads, exports every
function include/lbmdem.h declares, and its parameter struct matches the
Python mirror field by field.  No compute call is made (there is no GPU here).
"""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

from paper_1808_08921_gb300 import build, lbmdem

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbmdem.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_dem_\w+)\s*\(", txt)))


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    assert os.path.exists(path)
    lib = C.CDLL(path)
    declared = _declared()
    assert len(declared) >= 10
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(lbmdem.SYMBOLS) == declared


def test_params_struct_layout_matches_header():
    src = r"""
#include <stdio.h>
#include <stddef.h>
#include "lbmdem.h"
#define O(f) printf("%s %zu\n", #f, offsetof(lbmdem_params, f));
int main(void) {
  printf("size %zu\n", sizeof(lbmdem_params));
  O(nx) O(ny) O(nz) O(tau) O(rho_f) O(storage) O(inlet) O(outlet) O(dem_substeps)
  O(E_p) O(nu_p) O(mu) O(rho_p) O(body_force) O(probe_x) O(lbm_on) O(skin) O(dem_skin)
  O(monitor_every) O(graph_steps) O(max_flips) O(tile) O(device) O(cuda_stream)
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-I" + os.path.join(ROOT, "include"), c, "-o", exe])
        out = subprocess.check_output([exe], text=True).split("\n")
    got = dict(l.split() for l in out if l.strip())
    assert int(got.pop("size")) == C.sizeof(lbmdem.Params)
    for name, val in got.items():
        assert getattr(lbmdem.Params, name).offset == int(val), name


def test_default_params_and_argument_checks_without_gpu():
    lib = lbmdem.load()
    p = lbmdem.default_params()
    assert p.tau == 0.8 and p.dem_substeps == 10 and p.rho_p == 2.466 and p.probe_x == -1
    h = C.c_void_p()
    bad = lbmdem.default_params()
    bad.tau = 0.5  # Eq. 4 needs tau > 1/2
    assert lib.lbm_dem_init(C.byref(bad), C.byref(h)) == -1
    bad = lbmdem.default_params()
    bad.graph_steps = 3  # graphs hold an even number of steps
    assert lib.lbm_dem_init(C.byref(bad), C.byref(h)) == -1
    assert lib.lbm_dem_step(None, 1) == -1


@pytest.mark.parametrize("field,value", [
    ("nx", 0),            # a zero-length column
    ("nx", 2),            # a pressure inlet and an outlet need three planes
    ("probe_x", 128),     # probe plane outside the column (nx = 128)
    ("probe_x", -2),
    ("tau", float("nan")),
    ("rho_f", 0.0),
    ("dem_substeps", 0),
    ("storage", 7),
    ("inlet", 3),
    ("outlet", -1),
    ("nu_p", 0.5),        # Poisson ratio of Eqs. 11-12 below 1/2
    ("mu", -0.1),
    ("rho_p", 0.0),
    ("tile", 96),
    ("link_mode", 3),
    ("skin", -0.1),
    ("max_flips", -1),
])
def test_bad_parameters_are_refused_before_any_device_work(field, value):
    """Corrupt parameters come back as LBMDEM_ERR_INVALID_ARG from
    lbm_dem_init, with no context created (no GPU needed)."""
    lib = lbmdem.load()
    p = lbmdem.default_params()
    p.nx, p.ny, p.nz = 128, 16, 16
    setattr(p, field, value)
    h = C.c_void_p()
    assert lib.lbm_dem_init(C.byref(p), C.byref(h)) == -1
    assert not h.value


def test_oracle_is_not_linked_into_the_library():
    path = build.build()
    out = subprocess.check_output(["nm", "-D", "--defined-only", path], text=True)
    assert "orc_" not in out
