"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs, element by element.

Bars (FP32 arithmetic against FP64):
  * solid map: identical (an integer decision taken in FP64 on both sides);
  * density: |rho_gpu - rho_ref| <= 1e-4 rho_ref, and <= 1e-3 of the largest
    density deviation |rho_ref - rho_f| (the signal is ~1e-3 of rho);
  * velocity: |u_gpu - u_ref| <= 1e-4 max |u_ref|;
  * sphere centres within 1e-6 lattice units; hydrodynamic force and
    torque (Eqs. 18-19), velocity and angular velocity within 1e-3 of their
    largest component (torque also of R |F|, angular velocity of |V| / R);
    orientation quaternions within 1e-5.
"""
import math

import numpy as np
import pytest

import oracle
import workloads
from paper_1808_08921_gb300 import lbmdem

pytestmark = pytest.mark.gpu


def _sim(w, **over):
    return lbmdem.Sim.from_workload(w, **over)


def compare_fields(g, o, rho_f=1.0, sig_tol=1e-3):
    rg, ug, sg = g.fields()
    ro, uo, so = o.fields()
    assert np.array_equal(sg, so), f"solid maps differ at {np.argwhere(sg != so)[:5]}"
    fl = so == 0
    drho = np.abs(rg - ro)[fl]
    assert drho.max() <= 1e-4 * ro[fl].min()
    sig = np.abs(ro[fl] - rho_f).max()
    if sig > 0:
        assert drho.max() <= sig_tol * sig, (drho.max(), sig)
    umax = np.abs(uo).max()
    du = np.abs(ug - uo).max()
    assert du <= 1e-4 * umax + 1e-12, (du, umax)
    return drho.max(), du, sig, umax


def compare_particles(g, o, xtol=1e-6, ftol=1e-3, qtol=1e-5, R=None):
    """Torques are measured against R |F| and angular velocities against
    |V| / R as well as against themselves: where symmetry makes the oracle's
    torque vanish (a chain on the box axis) the GPU's FP32 link sums leave a
    round-off torque of that scale times 1e-7."""
    pg, po = g.particles(), o.particles()
    if len(po["X"]) == 0:
        return 0.0
    dx = np.abs(pg["X"] - po["X"]).max()
    assert dx <= xtol, dx
    Rm = 1.0 if R is None else float(np.max(R))
    scale = {"Fh": np.abs(po["Fh"]).max(), "V": np.abs(po["V"]).max()}
    scale["Th"] = max(np.abs(po["Th"]).max(), Rm * scale["Fh"])
    scale["W"] = max(np.abs(po["W"]).max(), scale["V"] / Rm)
    for k in ("Fh", "Th", "V", "W"):
        err = np.abs(pg[k] - po[k]).max()
        assert err <= ftol * scale[k] + 1e-12, (k, err, scale[k])
    assert np.abs(pg["q"] - po["q"]).max() <= qtol, np.abs(pg["q"] - po["q"]).max()
    return dx


@pytest.mark.parametrize("steps", [120, 121])
def test_pure_fluid_plane_wave(steps):
    w = workloads.plane_wave(nx=200, ny=2, nz=3, amplitude=1e-3, omega=0.05, steps=steps)
    g, o = _sim(w), oracle.Oracle(w)
    g.step(steps)
    o.step(steps)
    compare_fields(g, o)


@pytest.mark.parametrize("outlet", [workloads.OUTLET_ZERO_GRADIENT, workloads.OUTLET_PRESSURE,
                                    workloads.OUTLET_WALL])
def test_static_spheres_each_outlet(outlet):
    w = workloads.random_small(7, nx=30, ny=13, nz=37, n=4, R=3.3, tau=0.7, mobile=False)
    w.outlet = outlet
    w.amplitude, w.omega = 2e-3, 2 * math.pi / 40
    g, o = _sim(w), oracle.Oracle(w)
    for n in (1, 20, 39):
        g.step(n)
        o.step(n)
        compare_fields(g, o)
        compare_particles(g, o)


@pytest.mark.parametrize("seed,link_mode", [(1, 0), (4, 0), (1, 2)])
def test_moving_spheres_with_conversions(seed, link_mode):
    """Periodic box, spheres moving ~1 lu: nodes are covered and uncovered;
    the default link path and the even steps' links in the collide kernel
    (link words renewed at each conversion)."""
    w = workloads.random_small(seed, nx=22, ny=14, nz=12, n=3, R=3.1, tau=0.8, mobile=True, vel=0.05)
    w.inlet = workloads.X_PERIODIC
    w.rho_p, w.dem_substeps = 3.0, 3
    g, o = _sim(w, skin=0.6, dem_skin=1.2, link_mode=link_mode), oracle.Oracle(w)
    o0 = o.owner().copy()
    for n in (2, 17, 41):
        g.step(n)
        o.step(n)
        compare_fields(g, o)
        compare_particles(g, o)
    assert ((o.owner() >= 0) != (o0 >= 0)).sum() > 30
    assert g.counters()["conversions"] > 30


def test_parity_config_short():
    w = workloads.config_parity(steps=200)
    g, o = _sim(w), oracle.Oracle(w)
    for n in (1, 49, 150):
        g.step(n)
        o.step(n)
        compare_fields(g, o)
        compare_particles(g, o)


def test_parity_config_full_2000_steps():
    w = workloads.config_parity(steps=2000)
    g, o = _sim(w), oracle.Oracle(w)
    g.step(2000)
    o.step(2000)
    dr, du, sig, umax = compare_fields(g, o)
    dx = compare_particles(g, o)
    print(f"parity 2000 steps: |drho| {dr:.3e} (signal {sig:.3e}), |du| {du:.3e} "
          f"(max {umax:.3e}), |dX| {dx:.3e}")


def test_dem_only_oblique_collisions():
    rng = np.random.default_rng(3)
    X = np.array([[20, 20, 20], [29.7, 21.5, 20.5], [20.3, 29.8, 21], [30.5, 31, 19]], float)
    w = workloads.Workload(name="dem", nx=60, ny=40, nz=40, tau=1.0, mu=0.4, X=X,
                           R=np.full(4, 5.0), V=rng.uniform(-0.02, 0.02, (4, 3)),
                           W=rng.uniform(-0.003, 0.003, (4, 3)), fixed=np.zeros(4, np.uint8),
                           dem_substeps=10)
    g = lbmdem.Sim(lbmdem.params_from_workload(w, lbm_on=0, dem_skin=2.0))
    g.set_packing(w.X, w.R, w.V, w.W, w.fixed)
    o = oracle.Oracle(w, lbm_on=False)
    m = w.rho_p * 4 / 3 * math.pi * 125.0
    p0 = m * g.particles()["V"].sum(0)
    # through the first collisions: the 1e-6 lu bar
    g.step(60)
    o.step(60)
    pg, po = g.particles(), o.particles()
    assert np.abs(pg["X"] - po["X"]).max() < 1e-6
    assert np.abs(pg["V"] - po["V"]).max() < 1e-6 * np.abs(po["V"]).max()
    assert np.abs(pg["q"] - po["q"]).max() < 1e-5
    # repeated frictional collisions amplify FP32 rounding: a looser bar on
    # the trajectory, exact antisymmetry of the pair forces on the momentum
    g.step(90)
    o.step(90)
    pg, po = g.particles(), o.particles()
    assert np.abs(pg["X"] - po["X"]).max() < 1e-5
    assert np.abs(m * pg["V"].sum(0) - p0).max() < 1e-6 * m * np.abs(pg["V"]).sum()


def test_probe_trace_matches():
    w = workloads.config_parity(steps=60)
    w.probe_x = 41
    g, o = _sim(w), oracle.Oracle(w)
    g.step(60)
    o.step(60)
    pg, po = g.probe(), o.probe()
    assert len(pg) == len(po) == 60
    assert np.abs(pg - po).max() <= 1e-3 * np.abs(po - 1.0).max() + 1e-12


def test_pure_fluid_column_ragged_and_empty():
    w = workloads.Workload(name="empty", nx=9, ny=3, nz=33, tau=0.9, amplitude=5e-3,
                           omega=0.2, dem_substeps=2)
    g, o = _sim(w), oracle.Oracle(w)
    for n in (1, 1, 13):
        g.step(n)
        o.step(n)
        compare_fields(g, o)


def test_forced_relayout_keeps_the_state():
    """A re-layout only re-orders storage: fields before and after are equal,
    and the run continues in parity with the oracle."""
    w = workloads.random_small(1, nx=22, ny=14, nz=12, n=3, R=3.1, tau=0.8, mobile=True, vel=0.05)
    w.inlet = workloads.X_PERIODIC
    w.rho_p, w.dem_substeps = 3.0, 3
    g, o = _sim(w, skin=0.6, dem_skin=1.2), oracle.Oracle(w)
    g.step(4)
    o.step(4)
    r0, u0, s0 = g.fields()
    g.relayout()
    r1, u1, s1 = g.fields()
    assert np.array_equal(s0, s1)
    assert np.array_equal(r0, r1) and np.array_equal(u0, u1)
    g.step(9)
    o.step(9)
    compare_fields(g, o)
    compare_particles(g, o)


@pytest.mark.parametrize("workload", ["column", "plane_wave", "column_even_step"])
def test_fp64_monitors_match_oracle_totals(workload):
    """The FP64 totals the GPU accumulates on monitored steps (the drift
    monitor: sum rho and sum rho u over the fluid nodes, max |u|, Eq. 7) equal
    the oracle's sums over its fluid nodes of the same state.  A monitored
    step sums the state it starts from; with fixed spheres no node converts,
    so that is the oracle's state after the same number of completed steps.
    Graph-captured runs monitor their last (odd) step; five single steps
    with monitor_every = 5 monitor step 4, an even step, here with the
    step's links inside its collide kernel (link_mode 2)."""
    steps, every = 48, 16
    if workload == "plane_wave":
        w = workloads.plane_wave(nx=200, ny=2, nz=3, amplitude=1e-3, omega=0.05, steps=48)
    else:
        w = workloads.config_parity(steps=48)
        w.fixed = np.ones(len(w.R), np.uint8)
        if workload == "column_even_step":
            steps, every = 5, 5
    over = dict(link_mode=2) if workload == "column_even_step" else {}
    g, o = _sim(w, monitor_every=every, **over), oracle.Oracle(w)
    g.step(steps)
    mon = g.monitors()
    k = int(mon[5])
    assert k == steps - 1
    o.step(k)
    ro, uo, so = o.fields()
    fl = so == 0
    j = (uo * ro[None])[:, fl].sum(axis=1)
    assert abs(mon[0] - ro[fl].sum()) <= 1e-4 * np.abs(ro[fl] - w.rho_f).sum()
    jabs = np.abs(uo * ro[None])[:, fl].sum(axis=1)
    assert np.all(np.abs(mon[1:4] - j) <= 1e-4 * jabs + 1e-15), (mon[1:4], j)
    umax = np.sqrt((uo ** 2).sum(axis=0))[fl].max()
    assert abs(mon[4] - umax) <= 1e-4 * umax
