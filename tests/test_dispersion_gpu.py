"""Plane averages through the C ABI against the FP64 oracle's fields, and
the dispersion relation of the pure fluid from their space-time DFT: the
lattice sound speed 1/sqrt(3) is recovered (Section 3.2)."""
import math

import numpy as np
import pytest

import oracle
import workloads
from paper_1808_08921_gb300 import dispersion, lbmdem

pytestmark = pytest.mark.gpu


def test_plane_means_match_oracle():
    w = workloads.config_parity(steps=60)
    g = lbmdem.Sim.from_workload(w)
    o = oracle.Oracle(w)
    for n in (31, 29):  # both AA parities
        g.step(n)
        o.step(n)
        rho_g, jx_g = g.plane_means()
        rho, u, sol = o.fields()
        fl = sol == 0
        cnt = fl.sum(axis=(1, 2))
        rho_o = np.where(fl, rho, 0).sum(axis=(1, 2)) / cnt
        jx_o = np.where(fl, rho * u[0], 0).sum(axis=(1, 2)) / cnt
        sig = np.abs(rho_o - 1.0).max()
        assert np.abs(rho_g - rho_o).max() <= 1e-3 * sig
        assert np.abs(jx_g - jx_o).max() <= 1e-4 * np.abs(jx_o).max()


def test_dispersion_recovers_lattice_sound_speed():
    omega = 0.1
    w = workloads.plane_wave(nx=600, ny=2, nz=2, tau=1.0, amplitude=1e-4, omega=omega, t_n=100000, steps=1200)
    g = lbmdem.Sim.from_workload(w)
    st = dispersion.record(g, 1200, every=1)
    c = dispersion.phase_speed(st, omega)
    print(f"phase speed {c:.5f} (1/sqrt(3) = {1 / math.sqrt(3):.5f})")
    assert abs(c * math.sqrt(3) - 1) < 0.02
