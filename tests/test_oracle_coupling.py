"""Pins of the oracle's fluid-solid coupling (Section 2.3) and the wave
benchmark (Section 3.2).

* Static spheres in a closed box: the bounce-back of Eq. 14 with V_b = 0
  moves no mass, so total mass is conserved to round-off.
* Moving spheres in a fully periodic box: link exchange (Eq. 15) and the
  node conversions (Eqs. 16-17) move momentum between fluid and particles
  only.  The spheres are driven by the mean of the exchange sums of the
  current and previous step, so fluid + sphere momentum + half the last
  step's sum is conserved to round-off -- this fixes the signs of Eqs. 15-17
  and the lever-free parts of Eqs. 18-19.
* A translating and a rotating sphere feel the closed-form Stokes drag
  (Hasimoto's periodic-array correction for translation), which fixes the
  magnitude of the link force and the torque lever arms of Eq. 19.
* The plane wave of Eq. 27: absorption 7.79e-4 and speed 1/sqrt(3) at
  tau = 1, omega = 0.03 (golden values printed in Section 3.2).
"""
import math
import os

import numpy as np
import pytest
from scipy.optimize import curve_fit

import oracle
import workloads


def _fluid_momentum(s):
    c, _, _ = oracle.lattice()
    f = s.populations().reshape(19, -1)
    sol = s.owner().reshape(-1) >= 0
    f = f[:, ~sol]
    return np.einsum("mn,ma->a", f, c)


def _fluid_mass(s):
    f = s.populations().reshape(19, -1)
    sol = s.owner().reshape(-1) >= 0
    return f[:, ~sol].sum()


def test_closed_box_static_spheres_conserve_mass():
    w = workloads.random_small(3, nx=18, ny=11, nz=13, n=3, R=2.7, tau=0.65, mobile=False)
    w.inlet, w.outlet = workloads.X_WALL, workloads.OUTLET_WALL
    s = oracle.Oracle(w)
    rng = np.random.default_rng(5)
    f = s.populations()
    f = f + rng.uniform(-1e-3, 1e-3, f.shape)
    s.set_populations(f)
    m0 = _fluid_mass(s)
    s.step(60)
    assert abs(_fluid_mass(s) - m0) < 1e-11 * m0


def _periodic_moving(seed, steps):
    w = workloads.random_small(seed, nx=22, ny=14, nz=12, n=3, R=3.1, tau=0.8,
                               mobile=True, vel=0.05)
    w.inlet = workloads.X_PERIODIC
    w.rho_p = 3.0
    w.dem_substeps = 3
    return w


@pytest.mark.parametrize("seed", [1, 4])
def test_periodic_box_conserves_total_momentum(seed):
    w = _periodic_moving(seed, 80)
    s = oracle.Oracle(w)
    m = w.rho_p * 4 / 3 * math.pi * w.R ** 3

    def total():
        P = s.particles()
        return _fluid_momentum(s) + (m[:, None] * P["V"]).sum(0) + 0.5 * P["Fh"].sum(0)

    p0 = total()
    o0 = s.owner().copy()
    s.step(80)
    flipped = int(((s.owner() >= 0) != (o0 >= 0)).sum())
    assert flipped > 50  # many nodes covered and uncovered along the way
    assert np.allclose(total(), p0, atol=1e-11), (total(), p0)


def test_translating_sphere_stokes_drag():
    """Heavy free sphere at low Re in a periodic box: drag against the mean
    fluid velocity equals 6 pi eta R (V - u) times Hasimoto's periodic-array
    factor K = 1 / (1 - 1.7601 phi^(1/3) + phi - 1.5593 phi^2)."""
    L, R, tau, V0 = 24, 4.0, 0.8, 2e-3
    w = workloads.Workload(name="drag", nx=L, ny=L, nz=L, tau=tau, inlet=workloads.X_PERIODIC,
                           X=np.array([[L / 2 + 0.3, L / 2 + 0.2, L / 2 + 0.1]]),
                           R=np.array([R]), fixed=np.zeros(1, np.uint8),
                           V=np.array([[V0, 0, 0]]), W=np.zeros((1, 3)), rho_p=500.0,
                           dem_substeps=1, mu=0.0)
    s = oracle.Oracle(w)
    s.step(400)
    P = s.particles()
    rho, u, sol = s.fields()
    ubar = (rho * u[0]).sum() / rho[sol == 0].sum()
    eta = (tau - 0.5) / 3
    phi = 4 / 3 * math.pi * R ** 3 / L ** 3
    K = 1 / (1 - 1.7601 * phi ** (1 / 3) + phi - 1.5593 * phi ** 2)
    F_th = 6 * math.pi * eta * R * (P["V"][0, 0] - ubar) * K
    ratio = -P["Fh"][0, 0] / F_th
    assert 0.85 < ratio < 1.15, ratio
    # lateral force and torque vanish by symmetry (up to the staircase)
    assert abs(P["Fh"][0, 1]) < 0.05 * abs(P["Fh"][0, 0])


def test_rotating_sphere_stokes_torque():
    """Heavy spinning sphere: T = -8 pi eta R^3 Omega (unbounded Stokes)."""
    L, R, tau, W0 = 24, 4.0, 0.8, 1e-3
    w = workloads.Workload(name="spin", nx=L, ny=L, nz=L, tau=tau, inlet=workloads.X_PERIODIC,
                           X=np.array([[L / 2, L / 2, L / 2]]), R=np.array([R]),
                           fixed=np.zeros(1, np.uint8), V=np.zeros((1, 3)),
                           W=np.array([[0, 0, W0]]), rho_p=500.0, dem_substeps=1, mu=0.0)
    s = oracle.Oracle(w)
    s.step(300)
    P = s.particles()
    eta = (tau - 0.5) / 3
    ratio = -P["Th"][0, 2] / (8 * math.pi * eta * R ** 3 * P["W"][0, 2])
    assert 0.8 < ratio < 1.25, ratio
    assert abs(P["Th"][0, 0]) < 1e-3 * abs(P["Th"][0, 2])


def _golden(golden_dir, name):
    out = {}
    for l in open(os.path.join(golden_dir, name)):
        if l.strip() and not l.startswith("#"):
            k, v = l.split()
            out[k] = float(v)
    return out


def test_eq27_closed_form_reproduces_printed_alpha(golden_dir):
    g = _golden(golden_dir, "plane_wave.txt")
    cs = 1 / math.sqrt(3)
    nu = (g["tau"] - 0.5) * cs ** 2
    tau_s = 2 * nu / cs ** 2
    x2 = (g["omega"] * tau_s) ** 2
    alpha = g["omega"] / (cs * math.sqrt(2)) * math.sqrt((math.sqrt(1 + x2) - 1) / math.sqrt(1 + x2))
    assert abs(alpha - g["alpha_s"]) < 0.005 * g["alpha_s"]


def test_plane_wave_absorption_and_speed(golden_dir):
    """Section 3.2 benchmark: fit rho'(x) at t = 800 to Eq. 27."""
    g = _golden(golden_dir, "plane_wave.txt")
    w = workloads.plane_wave(tau=g["tau"], omega=g["omega"], amplitude=g["amplitude"],
                             steps=int(g["t_snapshot"]))
    s = oracle.Oracle(w)
    s.step(w.steps)
    rho, _, _ = s.fields()
    rp = rho.mean(axis=(1, 2)) - 1.0
    om, t = g["omega"], g["t_snapshot"]
    # fit window: behind the wave front (c_s t = 462) by a few wavelengths
    x = np.arange(20, 301).astype(float)

    def model(x, a, b, al, k):
        ph = om * t - k * x
        return np.exp(-al * x) * (a * np.cos(ph) - b * np.sin(ph))

    p, _ = curve_fit(model, x, rp[20:301] / g["amplitude"], p0=[0, -1, g["alpha_s"], om / g["c_s"]])
    assert abs(p[2] / g["alpha_s"] - 1) < 0.02
    assert abs(om / p[3] / g["c_s"] - 1) < 0.005
    assert abs(p[1] - g["A_im"]) < 0.02


def test_uncovered_nodes_take_neighbour_density():
    """Eq. 17: a node a sphere uncovers is rebuilt with the mean density of
    its fluid neighbours.  In a fluid at rho0 = 1.2 != rho_f the fluid mass
    then changes only by rho0 times the change of the staircase volume (plus
    the small pressure dipole of the slow sphere); rebuilding at rho_f, or
    averaging over solid neighbours too, misses this by ~0.2 per node."""
    w = workloads.Workload(name="m", nx=30, ny=16, nz=16, tau=0.8, inlet=workloads.X_PERIODIC,
                           X=np.array([[10.2, 8.1, 8.3]]), R=np.array([4.0]),
                           V=np.array([[0.01, 0.004, 0.0]]), W=np.array([[0, 0, 0.01]]),
                           fixed=np.zeros(1, np.uint8), rho_p=200.0, dem_substeps=1, mu=0.0)
    s = oracle.Oracle(w)
    s.set_populations(s.populations() * 1.2)
    m0, o0 = _fluid_mass(s), s.owner().copy()
    s.step(200)
    flips = int(((s.owner() >= 0) != (o0 >= 0)).sum())
    dN = int((s.owner() >= 0).sum() - (o0 >= 0).sum())
    assert flips > 100
    assert abs(_fluid_mass(s) - m0 + 1.2 * dN) < 0.01 * 1.2 * flips


@pytest.mark.parametrize("outlet,sign", [(workloads.OUTLET_PRESSURE, -1), (workloads.OUTLET_WALL, 1),
                                         (workloads.OUTLET_ZERO_GRADIENT, 0)])
def test_outlet_reflection(outlet, sign):
    """A one-period pulse reflects from the far end: a pressure-locked end
    (rho = rho_f, Section 3.2) returns it inverted, a resting wall returns it
    upright with the same magnitude, and the zero-gradient outlet returns
    much less.  Read at a probe plane (Section 3.2 averages over fluid)."""
    def run(out):
        w = workloads.plane_wave(nx=300, amplitude=1e-4, omega=2 * math.pi / 40, t_n=40, steps=0)
        w.tau, w.probe_x = 0.6, 100
        w.outlet = out
        s = oracle.Oracle(w)
        s.step(1150)
        tr = s.probe() - 1.0
        inc, ref = tr[:450], tr[750:]   # reflection returns near t = 870-960
        return inc[np.argmax(np.abs(inc))], ref[np.argmax(np.abs(ref))]
    inc_w, ref_w = run(workloads.OUTLET_WALL)
    inc, ref = run(outlet)
    assert abs(inc - inc_w) < 1e-15
    if sign == 0:
        assert abs(ref) < 0.35 * abs(ref_w)
    else:
        assert abs(ref - sign * ref_w) < 0.02 * abs(ref_w)
        assert abs(ref_w) > 0.3 * abs(inc)


def test_probe_matches_fields():
    """The probe is the fluid-node mean density of its plane entering a step."""
    w = workloads.config_parity(steps=30)
    w.probe_x = 37
    s = oracle.Oracle(w)
    s.step(29)
    rho, _, sol = s.fields()
    expect = rho[37][sol[37] == 0].mean()
    s.step(1)
    assert abs(s.probe()[-1] - expect) < 1e-15


def test_touching_spheres_share_the_contact_lens_symmetrically():
    """Two equal fixed spheres overlapping by 0.1, mirror-symmetric about the
    plane x = 14.5: each owns its own half of the contact lens (smallest
    |x - X|^2 / R^2).  Eq. 15 is counted about the rest state, so in a fluid
    at rest at rho_f the spheres feel no force at all, while at a uniform
    density rho_f + 0.2 the excess pressure presses on the wetted surfaces
    only and pushes the spheres together with mirror-image forces that scale
    with the excess (the same pair at rho_f + 0.4 feels twice the force)."""
    X = np.array([[10.55, 8.3, 8.2], [18.45, 8.3, 8.2]])

    def force(excess):
        w = workloads.Workload(name="lens", nx=29, ny=17, nz=17, tau=0.8, inlet=workloads.X_PERIODIC,
                               X=X, R=np.array([4.0, 4.0]), fixed=np.ones(2, np.uint8), dem_substeps=1)
        s = oracle.Oracle(w)
        own = s.owner()
        assert (own[:15] == 1).sum() == 0 and (own[15:] == 0).sum() == 0
        s.set_populations(s.populations() * (1.0 + excess))
        s.step(1)
        return s.particles()["Fh"]

    assert np.abs(force(0.0)).max() < 1e-12
    F1, F2 = force(0.2), force(0.4)
    assert abs(F1[0, 0] + F1[1, 0]) < 1e-12
    assert abs(F1[0, 1] - F1[1, 1]) < 1e-12 and abs(F1[0, 2] - F1[1, 2]) < 1e-12
    assert F1[0, 0] > 0.1
    assert abs(F2[0, 0] - 2 * F1[0, 0]) < 1e-9 * F1[0, 0]


@pytest.mark.parametrize("seed", [1, 4])
def test_moving_spheres_mass_budget(seed):
    """With moving spheres the fluid mass is not conserved, but its change
    over a step is fixed exactly: the moving-wall term of Eq. 14 adds
    -6 w_d rho_f c_d . V_b on every link, a covered node takes its mass out
    (Eq. 16) and an uncovered node brings rho_bar, the mean density of its
    neighbours that were fluid (Eq. 17).  The links, wall velocities and
    conversions are enumerated here from the owner maps and sphere states,
    independently of the oracle's own loops."""
    w = _periodic_moving(seed, 30)
    s = oracle.Oracle(w)
    c, wts, _ = oracle.lattice()
    shape = (w.nx, w.ny, w.nz)
    L = np.array(shape, float)
    s.step(3)
    checked_links = 0
    for _ in range(12):
        f = s.populations().reshape(19, *shape)
        rho = f.sum(axis=0)
        own0 = s.owner().reshape(shape)
        P = s.particles()
        m0 = rho[own0 < 0].sum()
        s.step(1)
        own1 = s.owner().reshape(shape)
        m1 = s.populations().reshape(19, *shape).sum(axis=0)[own1 < 0].sum()
        pred = m0
        cov = (own0 < 0) & (own1 >= 0)
        unc = (own0 >= 0) & (own1 < 0)
        pred -= rho[cov].sum()
        for x, y, z in zip(*np.nonzero(unc)):
            vals = []
            for m in range(18):
                q = ((x + c[m, 0]) % w.nx, (y + c[m, 1]) % w.ny, (z + c[m, 2]) % w.nz)
                if own0[q] < 0:
                    vals.append(rho[q])
            pred += np.mean(vals) if vals else w.rho_f
        # links of the step: fluid node x, solid neighbour x + c_d (map of the step)
        fl = np.argwhere(own1 < 0)
        for m in range(18):
            nb = (fl + c[m]) % np.array(shape)
            p = own1[nb[:, 0], nb[:, 1], nb[:, 2]]
            sel = p >= 0
            if not sel.any():
                continue
            xb = fl[sel] + 0.5 * c[m]
            pid = p[sel]
            r = xb - P["X"][pid]
            r -= L * np.round(r / L)
            vb = P["V"][pid] + np.cross(P["W"][pid], r)
            pred -= (6.0 * wts[m] * w.rho_f * (vb @ c[m])).sum()
            checked_links += int(sel.sum())
        assert abs(m1 - pred) < 1e-11 * m0, (m1 - pred, m1 - m0)
    assert checked_links > 1000


def _d3q19(golden_dir):
    """c[19, 3] from the printed columns of Eq. 3 and the weights of Eq. 8."""
    rows = [list(map(int, l.split())) for l in open(os.path.join(golden_dir, "d3q19_velocities.txt"))
            if l.strip() and not l.startswith("#")]
    c = np.array(rows).T
    c2 = (c * c).sum(1)
    return c, np.where(c2 == 0, 1 / 3, np.where(c2 == 1, 1 / 18, 1 / 36))


def test_link_momentum_rest_state_equals_literal_on_a_wetted_sphere():
    """Reading of Eq. 15: the link momentum is counted about the rest state,
    c_d (f~_d + f_d* - 2 w_d rho_f), instead of the printed c_d (f~_d + f_d*).
    The two differ by 2 rho_f sum_links w_d c_d (and its moment), which is
    zero over the closed staircase of a sphere whose every neighbour node is
    fluid: so a moving, spinning sphere alone in a periodic box feels the
    same force and torque under both forms, step after step (and, since
    that drives it, follows the same path)."""
    w = workloads.Workload(name="wet", nx=24, ny=22, nz=21, tau=0.8, inlet=workloads.X_PERIODIC,
                           X=np.array([[11.3, 10.6, 9.9]]), R=np.array([4.6]),
                           V=np.array([[0.012, -0.007, 0.004]]), W=np.array([[0.002, 0.0015, -0.003]]),
                           fixed=np.zeros(1, np.uint8), rho_p=2.0, dem_substeps=2)
    a, b = oracle.Oracle(w), oracle.Oracle(w)
    b.set_link_form(True)
    for _ in range(6):
        a.step(5)
        b.step(5)
        pa, pb = a.particles(), b.particles()
        assert np.abs(pa["Fh"]).max() > 1e-4          # a real drag, not zero
        assert np.abs(pa["Fh"] - pb["Fh"]).max() < 1e-12
        assert np.abs(pa["Th"] - pb["Th"]).max() < 1e-12
        assert np.abs(pa["X"] - pb["X"]).max() < 1e-13
    # the staircase moved: nodes were covered and uncovered on the way
    assert a.t == 30


def test_link_momentum_forms_differ_by_the_dry_contact_caps(golden_dir):
    """On two touching spheres the two readings of Eq. 15 differ, for sphere
    p, by exactly -2 rho_f sum w_d c_d over the node pairs (s, s - c_d) with
    s owned by p and s - c_d owned by the other sphere -- the dry contact
    caps -- and the torque by the moment of those terms about X_p at the
    link midpoint s - c_d / 2.  The pairs are enumerated here from the owner
    map and the printed velocity set, independently of the oracle's loops;
    the spheres are fixed, so both runs share every population."""
    c, wts = _d3q19(golden_dir)
    X = np.array([[9.62, 8.41, 7.93], [17.03, 9.26, 9.48]])
    R = np.array([4.2, 3.9])
    w = workloads.Workload(name="lens2", nx=27, ny=18, nz=17, tau=0.75, inlet=workloads.X_PERIODIC,
                           X=X, R=R, fixed=np.ones(2, np.uint8), dem_substeps=1)
    a, b = oracle.Oracle(w), oracle.Oracle(w)
    b.set_link_form(True)
    rng = np.random.default_rng(11)
    f = a.populations() * (1.0 + rng.uniform(-2e-3, 2e-3, a.populations().shape))
    a.set_populations(f)
    b.set_populations(f)
    own = a.owner()
    shape = np.array(own.shape)
    L = shape.astype(float)
    a.step(3)
    b.step(3)
    dF, dT = np.zeros((2, 3)), np.zeros((2, 3))
    npairs = 0
    for p, q in ((0, 1), (1, 0)):
        S = np.argwhere(own == p)
        for m in range(18):
            nb = (S - c[m]) % shape
            sel = own[nb[:, 0], nb[:, 1], nb[:, 2]] == q
            if not sel.any():
                continue
            npairs += int(sel.sum())
            term = -2.0 * w.rho_f * wts[m] * c[m]
            mid = S[sel] - 0.5 * c[m] - X[p]
            mid -= L * np.round(mid / L)
            dF[p] += sel.sum() * term
            dT[p] += np.cross(mid, term).sum(0)
    assert npairs > 10
    Fa, Fb = a.particles()["Fh"], b.particles()["Fh"]
    Ta, Tb = a.particles()["Th"], b.particles()["Th"]
    assert np.abs(dF).max() > 1e-3
    assert np.abs((Fb - Fa) - dF).max() < 1e-12, (Fb - Fa, dF)
    assert np.abs((Tb - Ta) - dT).max() < 1e-11, (Tb - Ta, dT)


def test_oracle_threads_do_not_change_results():
    """The oracle's OpenMP loops (x-planes) form every sum in one fixed order,
    so one thread and several give bit-identical populations and spheres on a
    case with moving spheres, node conversions and a contact."""
    w = workloads.random_small(11, nx=24, n=5, vel=0.02, steps=12)
    w.X[1] = w.X[0] + np.array([0.0, 2 * w.R[0] - 0.05, 0.0])   # one overlapping pair
    w.X[1, 1] %= w.ny
    runs = []
    before = oracle.threads()
    try:
        for n in (1, 3):
            oracle.set_threads(n)
            o = oracle.Oracle(w)
            o.step(12)
            runs.append((o.populations(), o.particles()))
    finally:
        oracle.set_threads(before)
    assert np.array_equal(runs[0][0], runs[1][0])
    for k in runs[0][1]:
        assert np.array_equal(runs[0][1][k], runs[1][1][k]), k
