"""Pins of the oracle's fluid core: D3Q19 tables, equilibrium, BGK, Zou-He.

Each check is fixed by the paper or by mathematics, not by the oracle:
the velocity matrix of Eq. 3 (golden file), lattice isotropy of the
weights of Eq. 8, the exact low-order moments of the equilibrium of Eq. 6,
mass/momentum conservation and the relaxation factor of Eq. 4, and the
moment identities of the pressure boundary of Section 2.4.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
import workloads


def _golden_c(golden_dir):
    rows = [list(map(int, l.split())) for l in open(os.path.join(golden_dir, "d3q19_velocities.txt"))
            if l.strip() and not l.startswith("#")]
    return np.array(rows).T


def test_velocity_set_matches_eq3(golden_dir):
    c, w, opp = oracle.lattice()
    assert np.array_equal(c, _golden_c(golden_dir))


def test_opposites_and_weights():
    c, w, opp = oracle.lattice()
    assert np.array_equal(c[opp], -c)
    assert np.array_equal(opp[opp], np.arange(19))
    # Eq. 8 by speed class
    for m in range(19):
        s = int((c[m] ** 2).sum())
        assert w[m] == {0: 1 / 3, 1: 1 / 18, 2: 1 / 36}[s]


def test_weight_isotropy():
    """sum w = 1, sum w c_a c_b = d_ab / 3, 4th moment = (dd + dd + dd) / 9."""
    c, w, _ = oracle.lattice()
    assert abs(w.sum() - 1) < 1e-15
    assert np.allclose(np.einsum("m,ma->a", w, c), 0, atol=1e-16)
    assert np.allclose(np.einsum("m,ma,mb->ab", w, c, c), np.eye(3) / 3, atol=1e-16)
    assert np.allclose(np.einsum("m,ma,mb,mc->abc", w, c, c, c), 0, atol=1e-16)
    d = np.eye(3)
    iso4 = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
            + np.einsum("ad,bc->abcd", d, d)) / 9
    assert np.allclose(np.einsum("m,ma,mb,mc,md->abcd", w, c, c, c, c), iso4, atol=1e-16)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_equilibrium_moments(seed):
    """Eq. 6 recovers rho, rho u and rho/3 I + rho u u exactly."""
    rng = np.random.default_rng(seed)
    c, _, _ = oracle.lattice()
    rho = rng.uniform(0.9, 1.1)
    u = rng.uniform(-0.05, 0.05, 3)
    feq = oracle.equilibrium(rho, u)
    assert abs(feq.sum() - rho) < 1e-14
    assert np.allclose(feq @ c, rho * u, atol=1e-15)
    Pi = np.einsum("m,ma,mb->ab", feq, c, c)
    assert np.allclose(Pi, rho / 3 * np.eye(3) + rho * np.outer(u, u), atol=1e-15)


@pytest.mark.parametrize("tau", [0.55, 0.8, 1.0, 1.7])
def test_bgk_conserves_and_relaxes(tau):
    """Eq. 4: mass and momentum conserved, non-equilibrium part scaled by 1 - 1/tau."""
    rng = np.random.default_rng(7)
    c, _, _ = oracle.lattice()
    f = oracle.equilibrium(1.0, [0.01, -0.02, 0.005]) + rng.uniform(-1e-3, 1e-3, 19)
    rho, j = f.sum(), f @ c
    ft = oracle.collide_node(f, tau)
    assert abs(ft.sum() - rho) < 1e-15
    assert np.allclose(ft @ c, j, atol=1e-16)
    feq = oracle.equilibrium(rho, j / rho)
    assert np.allclose(ft - feq, (1 - 1 / tau) * (f - feq), atol=1e-16)
    assert np.allclose(oracle.collide_node(feq, tau), feq, atol=1e-16)


@pytest.mark.parametrize("side", [0, 1])
def test_pressure_face_moments(side):
    """Section 2.4: after the boundary, sum f = rho_b and the two tangential
    momenta vanish; the normal momentum is what the mass balance leaves."""
    rng = np.random.default_rng(11 + side)
    c, _, _ = oracle.lattice()
    for _ in range(20):
        f = oracle.equilibrium(1.0, rng.uniform(-0.02, 0.02, 3)) + rng.uniform(-1e-3, 1e-3, 19)
        rb = 1 + rng.uniform(-1e-3, 1e-3)
        g = oracle.pressure_face(f, rb, side)
        assert abs(g.sum() - rb) < 1e-15
        assert abs(g @ c[:, 1]) < 1e-16 and abs(g @ c[:, 2]) < 1e-16
        # only the unknown populations (those entering the domain) change
        unknown = c[:, 0] == (1 if side == 0 else -1)
        assert np.array_equal(g[~unknown], f[~unknown])


@pytest.mark.parametrize("side", [0, 1])
def test_pressure_face_equilibrium_fixed_point(side):
    """Non-equilibrium bounce-back is exact for an equilibrium state with
    zero tangential velocity: the rebuilt unknowns equal f^eq."""
    for ux in (-0.03, 0.0, 0.02):
        feq = oracle.equilibrium(1.0007, [ux, 0, 0])
        c, _, _ = oracle.lattice()
        unknown = c[:, 0] == (1 if side == 0 else -1)
        f = feq.copy()
        f[unknown] = 0.123
        g = oracle.pressure_face(f, 1.0007, side)
        assert np.allclose(g, feq, atol=1e-15)


def test_source_waveforms():
    """Eq. 25 and Table 2: sine, cosine (1 - cos), step; rho_f after t_n."""
    w = workloads.plane_wave()
    w.amplitude, w.omega, w.t_n = 2e-3, 0.1, 50
    for wf, fn in [(workloads.SINE, lambda t: math.sin(0.1 * t)),
                   (workloads.COSINE, lambda t: 1 - math.cos(0.1 * t)),
                   (workloads.STEP, lambda t: 1.0)]:
        w.waveform = wf
        s = oracle.Oracle(w)
        for t in (0, 1, 17, 50):
            assert abs(s.source_density(t) - (1 + 2e-3 * fn(t))) < 1e-15
        assert s.source_density(51) == 1.0


def test_source_waveform_properties():
    """Eq. 25's source shapes pinned by what each waveform is for rather
    than by its formula: the sine starts at zero rising and its spectrum peaks
    at omega / 2 pi; the 1 - cos ramp starts at zero with zero slope (the
    smooth start), never goes below the background, peaks at 2 rho' after
    half a period and averages rho' over whole periods; the step holds
    rho' from t = 0 to t_n.  A cos for 1 - cos, a sin/cos swap or omega read
    as a frequency in cycles per step fails one of these."""
    amp, period = 1e-3, 64.0
    w = workloads.plane_wave()
    w.amplitude, w.omega, w.t_n = amp, 2 * math.pi / period, -1
    T = np.arange(0, 64 * 64)

    def shape(wf):
        w.waveform = wf
        s = oracle.Oracle(w)
        return np.array([s.source_density(int(t)) - 1.0 for t in T]) / amp

    sn = shape(workloads.SINE)
    assert sn[0] == 0.0 and sn[1] > 0.0
    spec = np.abs(np.fft.rfft(sn))
    assert abs(np.fft.rfftfreq(len(T))[spec.argmax()] - 1.0 / period) < 1e-12
    assert abs(sn.sum()) < 1e-9
    cs = shape(workloads.COSINE)
    assert cs[0] == 0.0 and cs.min() >= 0.0
    assert cs[1] < 0.01 * cs[int(period / 4)]             # zero slope at the start
    assert abs(cs[int(period / 2)] - 2.0) < 1e-12 and cs.argmax() == int(period / 2)
    assert abs(cs.mean() - 1.0) < 1e-12
    st = shape(workloads.STEP)
    assert np.all(np.abs(st - 1.0) < 1e-12)
    w.t_n = 100
    assert abs(shape(workloads.STEP)[100] - 1.0) < 1e-12 and shape(workloads.STEP)[101] == 0.0


def test_ricker_pulse_shape():
    """The Ricker pulse (the sweep's added waveform, not in Table 2):
    r(t) = (1 - 2 a^2) exp(-a^2), a = pi f (t - t0), f = omega / 2 pi.  Pinned
    by what the standard wavelet fixes and the formula alone does not give
    away: its peak value at t0, zero crossings at a = +-1/sqrt(2), minima of
    -2 exp(-3/2) at a = +-sqrt(3/2), zero time integral, and an amplitude
    spectrum f'^2 exp(-f'^2 / f^2) that peaks at the peak frequency f.  A
    wrong factor in a (2 pi, pi or 1/2 misplaced) moves the crossings and
    the spectral peak; a wrong sign breaks the peak value."""
    period, t0, amp = 200.0, 400.0, 2e-3
    f = 1.0 / period
    w = workloads.plane_wave()
    w.waveform, w.amplitude, w.omega, w.t0, w.t_n = workloads.RICKER, amp, 2 * math.pi * f, t0, -1
    s = oracle.Oracle(w)
    T = np.arange(0, 4096)
    r = np.array([s.source_density(int(t)) - 1.0 for t in T]) / amp
    assert abs(r[int(t0)] - 1.0) < 1e-15 and r.argmax() == int(t0)
    tz = 1.0 / (math.sqrt(2.0) * math.pi * f)          # zero crossing offset
    for side in (-1, 1):
        a, b = int(math.floor(t0 + side * tz)), int(math.ceil(t0 + side * tz))
        assert r[a] * r[b] < 0, (side, r[a], r[b])
        tm = t0 + side * math.sqrt(1.5) / (math.pi * f)  # minimum
        k = int(round(tm))
        assert abs(r[k] + 2 * math.exp(-1.5)) < 1e-3
        assert r[k] <= r[k - 1] + 1e-3 and r[k] <= r[k + 1] + 1e-3
    assert abs(r.sum()) < 1e-9 * period                 # zero integral (smooth, decayed)
    spec = np.abs(np.fft.rfft(r, 1 << 18))
    fr = np.fft.rfftfreq(1 << 18)
    assert abs(fr[spec.argmax()] - f) < 0.01 * f
    # switched off after t_n like every other source
    w.t_n = 300
    s2 = oracle.Oracle(w)
    assert s2.source_density(301) == 1.0 and s2.source_density(300) != 1.0


def test_uniform_flow_is_fixed_point():
    """A uniform equilibrium flow in a fully periodic box never changes."""
    w = workloads.Workload(name="u", nx=6, ny=5, nz=4, tau=0.7, inlet=workloads.X_PERIODIC,
                           steps=5, dem_substeps=1)
    s = oracle.Oracle(w)
    f0 = np.repeat(oracle.equilibrium(1.01, [0.02, -0.01, 0.03])[:, None], w.nodes, 1)
    s.set_populations(f0)
    s.step(7)
    assert np.allclose(s.populations().reshape(19, -1), f0, atol=1e-15)


def test_streaming_shifts_each_population_by_c():
    """Eq. 5: with tau = 1 the post-collision state of a node is its own
    equilibrium, so one node carrying f^eq(rho, u) in a uniform rest state
    must deliver population m, unchanged, to node x + c_m (periodic)."""
    c, w, _ = oracle.lattice()
    wl = workloads.Workload(name="s", nx=7, ny=6, nz=5, tau=1.0, inlet=workloads.X_PERIODIC,
                            steps=1, dem_substeps=1)
    s = oracle.Oracle(wl)
    base = oracle.equilibrium(1.0, [0, 0, 0])
    f = np.repeat(base[:, None], wl.nodes, 1).reshape(19, 7, 6, 5)
    node_feq = oracle.equilibrium(1.02, [0.01, 0.02, -0.03])
    f[:, 3, 2, 1] = node_feq
    s.set_populations(f)
    s.step(1)
    g = s.populations()
    for m in range(19):
        x, y, z = (3 + c[m, 0]) % 7, (2 + c[m, 1]) % 6, (1 + c[m, 2]) % 5
        # tau = 1: post-collision = equilibrium of that node
        assert abs(g[m, x, y, z] - node_feq[m]) < 1e-15
