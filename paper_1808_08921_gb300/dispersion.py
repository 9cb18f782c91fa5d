"""Dispersion relation from space-time data (Section 3.2: the discrete
Fourier transform of the plane-averaged field over time and the propagation
direction gives omega(k); the slope through the driven frequency gives the
wave speed).

    st = record(sim, steps, every=1)        # [samples, nx] plane means of rho u_x
    k, w, power = spectrum(st, dt=every)
    c = phase_speed(st, omega_0, dt=every)  # speed at the driven frequency
"""
from __future__ import annotations

import numpy as np


def record(sim, steps, every=1, field="jx", x0=0, x1=None):
    """Step `sim` and sample the plane means of `field` ("rho" or "jx") every
    `every` steps; returns [steps // every, x1 - x0]."""
    out = []
    for _ in range(steps // every):
        sim.step(every)
        rho, jx = sim.plane_means()
        v = rho - np.nanmean(rho) if field == "rho" else jx
        out.append(np.nan_to_num(v[x0:x1]))
    return np.array(out)


def spectrum(st, dt=1.0, dx=1.0):
    """|F(k, omega)|^2 of the mean-removed space-time array (time along axis
    0, x along axis 1), with angular frequencies and wavenumbers (rad per
    step and per lattice unit, non-negative halves)."""
    a = st - st.mean()
    F = np.fft.rfft2(a * np.hanning(a.shape[0])[:, None] * np.hanning(a.shape[1])[None, :])
    # rfft2 halves the last axis (x); fold the time axis to |omega|
    P = np.abs(F) ** 2
    w = 2 * np.pi * np.fft.fftfreq(a.shape[0], dt)
    k = 2 * np.pi * np.fft.rfftfreq(a.shape[1], dx)
    return k, w, P


def phase_speed(st, omega0, dt=1.0, dx=1.0):
    """Wave speed at the driven angular frequency omega0: omega0 / k of the
    strongest wavenumber in the frequency row nearest omega0 (a wave running
    to +x appears at omega < 0 in the numpy sign convention)."""
    k, w, P = spectrum(st, dt, dx)
    row = int(np.argmin(np.abs(w + omega0)))
    j = int(np.argmax(P[row, 1:])) + 1
    # parabolic refinement of the peak
    if 1 <= j < len(k) - 1:
        y0, y1, y2 = np.log(P[row, j - 1:j + 2] + 1e-300)
        den = y0 - 2 * y1 + y2
        dj = 0.5 * (y0 - y2) / den if den != 0 else 0.0
    else:
        dj = 0.0
    kk = (j + dj) * (k[1] - k[0])
    return omega0 / kk
