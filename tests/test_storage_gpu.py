"""Populations stored as 16-bit deviations f_i - w_i rho_f (BF16, or FP16
scaled by 2^12), collided in FP32: the error against the FP64 oracle on the
16 x 16 x 128 column, next to the FP32 storage's, through the C ABI.

A stored deviation is rounded once per step, to 8 (BF16) or 11 (FP16)
significant bits; over the 2000-step run the rounding errors add up like a
random walk.  The bars are a few times the measured errors (FP16: density
3e-4 of the density signal rho', velocity 3e-2 of max |u|, centres 5e-8
lu), so they state the precision and catch regressions; the solid maps
must agree exactly.
"""
import numpy as np
import pytest

import oracle
import workloads
from paper_1808_08921_gb300 import lbmdem

pytestmark = pytest.mark.gpu

# fraction of the density signal, of max |u|, and lattice units for X
BARS = {lbmdem.F32: (1e-3, 1e-4, 1e-6),
        lbmdem.F16_DEV: (2e-3, 1e-1, 1e-6),
        lbmdem.BF16_DEV: (2e-2, 5e-1, 1e-5)}


def _errors(g, o):
    rg, ug, sg = g.fields()
    ro, uo, so = o.fields()
    fl = so == 0
    sig = np.abs(ro[fl] - 1.0).max()
    umax = np.abs(uo).max()
    pg, po = g.particles(), o.particles()
    return (bool(np.array_equal(sg, so)), np.abs(rg - ro)[fl].max() / sig, np.abs(ug - uo).max() / umax,
            np.abs(pg["X"] - po["X"]).max())


@pytest.fixture(scope="module")
def reference():
    w = workloads.config_parity(steps=2000)
    o = oracle.Oracle(w)
    snaps = {}
    for n in (200, 1800):
        o.step(n)
        rho, u, sol = o.fields()
        snaps[o.t] = (rho, u, sol, o.particles())
    return w, snaps


class _Snap:
    def __init__(self, s):
        self.s = s

    def fields(self):
        return self.s[0], self.s[1], self.s[2]

    def particles(self):
        return self.s[3]


@pytest.mark.parametrize("storage,link_mode", [(lbmdem.F32, 0), (lbmdem.F16_DEV, 0), (lbmdem.BF16_DEV, 0),
                                               (lbmdem.F32, 2), (lbmdem.F16_DEV, 2), (lbmdem.BF16_DEV, 2)])
def test_storage_error_against_oracle(reference, storage, link_mode):
    """link_mode 0: the default path (the link kernel every step here: the
    column's spheres have R 5.7); 2: an even step's links inside its collide
    kernel, on FP32 and on 16-bit populations."""
    w, snaps = reference
    g = lbmdem.Sim.from_workload(w, storage=storage, link_mode=link_mode)
    done = 0
    for t in sorted(snaps):
        g.step(t - done)
        done = t
        same, drho, du, dx = _errors(g, _Snap(snaps[t]))
        print(f"storage {storage} t {t}: |drho|/rho' {drho:.2e}  |du|/umax {du:.2e}  |dX| {dx:.2e} lu")
        br, bu, bx = BARS[storage]
        assert same, "solid maps differ"
        assert drho <= br and du <= bu and dx <= bx, (drho, du, dx)
    g.close()


@pytest.mark.parametrize("storage,link_mode", [(lbmdem.F16_DEV, 0), (lbmdem.BF16_DEV, 0), (lbmdem.F16_DEV, 2)])
def test_16bit_storage_through_conversions_and_relayout(storage, link_mode):
    """Spheres moving ~1 lu in a periodic box (nodes covered and uncovered,
    16-bit gather/scatter of the conversions) and a forced re-layout (the
    stored 16-bit populations move without conversion)."""
    w = workloads.random_small(1, nx=22, ny=14, nz=12, n=3, R=3.1, tau=0.8, mobile=True, vel=0.05)
    w.inlet = workloads.X_PERIODIC
    w.rho_p, w.dem_substeps = 3.0, 3
    g = lbmdem.Sim.from_workload(w, skin=0.6, dem_skin=1.2, storage=storage, link_mode=link_mode)
    o = oracle.Oracle(w)
    g.step(20)
    o.step(20)
    r0, u0, s0 = g.fields()
    g.relayout()
    r1, u1, s1 = g.fields()
    assert np.array_equal(s0, s1) and np.array_equal(r0, r1) and np.array_equal(u0, u1)
    g.step(21)
    o.step(21)
    assert g.counters()["conversions"] > 30
    same, drho, du, dx = _errors(g, o)
    print(f"storage {storage} moving: |drho|/rho' {drho:.2e}  |du|/umax {du:.2e}  |dX| {dx:.2e} lu")
    assert same
    br, bu, bx = BARS[storage]
    assert drho <= 10 * br and du <= bu and dx <= 10 * bx
