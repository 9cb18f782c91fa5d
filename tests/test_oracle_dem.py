"""Pins of the oracle's DEM (Section 2.2, Eqs. 9-12).

* Hertz normal force of Eq. 11 in closed form; the elastic tangential
  increment of Eq. 12; the Coulomb cap reached exactly under imposed
  sliding; the stored tangential force rotated into the new tangent plane.
* Head-on collision of two free spheres (no damping in Eqs. 11-12): the
  rebound speed equals the approach speed and the contact lasts the Hertz
  time 2 delta_max / v * int_0^1 (1 - x^{5/2})^{-1/2} dx.
* A sphere touching two periodic images of a neighbour feels the sum of
  both Hertz forces (a minimum-image search would miss one).
* Free flight is exact; a torque-free spinning sphere's quaternion follows
  the exact rotation; fixed spheres stay put; total momentum is conserved
  through a multi-sphere oblique frictional collision.
* The dry granular chain of Section 3.2 (60 spheres compressed by 0.01 at
  every contact, free ends): behind the rarefaction that runs in from each
  end the spheres move at the simple-wave speed of the Hertz law,
  (4/5) sqrt(1.5 k_n sqrt(R*)/m) delta_0^(5/4).
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad

import oracle
import workloads

KN = 2 * workloads.E_P / (3 * (1 - workloads.NU_P ** 2))
KT = 2 * workloads.E_P / ((1 + workloads.NU_P) * (2 - workloads.NU_P))


def _params(mu=0.3):
    return workloads.Workload(name="p", nx=8, ny=8, nz=8, tau=1.0, mu=mu)


@pytest.mark.parametrize("Ri,Rj,delta", [(5.0, 5.0, 0.01), (5.7, 3.2, 0.2), (11.4, 11.4, 0.173)])
def test_hertz_normal_closed_form(Ri, Rj, delta):
    n = np.array([1.0, 2.0, -0.5])
    n /= np.linalg.norm(n)
    d = n * (Ri + Rj - delta)
    F, h, ov = oracle.pair_force(_params(), Ri, Rj, d, np.zeros(3), 0.1, np.zeros(3))
    Rs = Ri * Rj / (Ri + Rj)
    assert abs(ov - delta) < 1e-12
    assert np.allclose(F, -KN * math.sqrt(Rs * delta) * delta * n, rtol=1e-12, atol=1e-15)
    assert np.allclose(h, 0)


def test_tangential_increment_and_cap():
    Ri = Rj = 5.0
    delta = 0.05
    d = np.array([0, 0, Ri + Rj - delta])
    Rs = 2.5
    fn = KN * math.sqrt(Rs * delta) * delta
    # small sliding of j along +x: elastic increment, friction on i along +x
    dt, v = 0.1, 1e-4
    F, h, _ = oracle.pair_force(_params(), Ri, Rj, d, np.array([v, 0, 0]), dt, np.zeros(3))
    assert np.allclose(h, [KT * math.sqrt(Rs * delta) * v * dt, 0, 0], rtol=1e-12)
    assert abs(F[2] + fn) < 1e-12 and abs(F[0] - h[0]) < 1e-15
    # large sliding: |F_t| capped at mu |F_n| exactly, along the slip
    F, h, _ = oracle.pair_force(_params(0.3), Ri, Rj, d, np.array([1.0, 1.0, 0]), dt, np.zeros(3))
    assert abs(np.linalg.norm(h) - 0.3 * fn) < 1e-12
    assert np.allclose(h / np.linalg.norm(h), [1 / math.sqrt(2), 1 / math.sqrt(2), 0])
    # history rotated into the new tangent plane (normal part removed)
    d2 = np.array([0.3, 0, Ri + Rj - delta])
    F2, h2, _ = oracle.pair_force(_params(0.3), Ri, Rj, d2, np.zeros(3), dt, h)
    n2 = d2 / np.linalg.norm(d2)
    assert abs(h2 @ n2) < 1e-15


def _dem_only(X, R, V=None, W=None, fixed=None, ny=40, nz=40, nx=60, K=10, mu=0.3):
    n = len(R)
    w = workloads.Workload(name="dem", nx=nx, ny=ny, nz=nz, tau=1.0, mu=mu,
                           X=np.array(X, float), R=np.array(R, float),
                           V=None if V is None else np.array(V, float),
                           W=None if W is None else np.array(W, float),
                           fixed=np.zeros(n, np.uint8) if fixed is None else np.array(fixed, np.uint8),
                           dem_substeps=K)
    return oracle.Oracle(w, lbm_on=False), w


def test_head_on_collision_hertz_time_and_elastic_rebound():
    R, v = 5.0, 0.01
    s, w = _dem_only([[20, 20, 20], [30.5, 20, 20]], [R, R], V=[[v / 2, 0, 0], [-v / 2, 0, 0]], K=20)
    m = w.rho_p * 4 / 3 * math.pi * R ** 3
    mstar = m / 2
    Kh = KN * math.sqrt(R / 2)
    dmax = (5 * mstar * v ** 2 / (4 * Kh)) ** 0.4
    I, _ = quad(lambda x: 1 / math.sqrt(1 - x ** 2.5), 0, 1)
    tc = 2 * dmax / v * I
    gaps = []
    for _ in range(200):
        s.step(1)
        X = s.particles()["X"]
        gaps.append(2 * R - (X[1, 0] - X[0, 0]))
    g = np.array(gaps)
    inside = np.nonzero(g > 0)[0]
    a, b = inside[0], inside[-1]
    t_in = a - g[a] / (g[a] - g[a - 1])       # linear interpolation of the crossings
    t_out = b + g[b] / (g[b] - g[b + 1])
    assert abs((t_out - t_in) / tc - 1) < 0.01
    V = s.particles()["V"]
    assert abs(V[0, 0] + v / 2) < 1e-5 * v and abs(V[1, 0] - v / 2) < 1e-5 * v
    assert abs(np.max(g) / dmax - 1) < 0.01


def test_two_periodic_images_both_act():
    """j sits 4.8 above i and 5.2 below through the periodic y boundary."""
    R = 3.0
    s, w = _dem_only([[10, 0.5, 5], [10, 5.3, 5]], [R, R], ny=10, nz=10, nx=20)
    Fc, _ = s.contact_forces()
    Rs = R / 2
    f_up = KN * math.sqrt(Rs * 1.2) * 1.2    # j at +4.8
    f_dn = KN * math.sqrt(Rs * 0.8) * 0.8    # j's image at -5.2
    assert abs(Fc[0, 1] - (-f_up + f_dn)) < 1e-12
    assert np.allclose(Fc[0], -Fc[1], atol=1e-14)


def test_free_flight_spin_and_fixed():
    W = np.array([0.01, -0.02, 0.015])
    s, w = _dem_only([[10, 10, 10], [40, 30, 30]], [3.0, 3.0],
                     V=[[0.013, -0.007, 0.002], [0.1, 0.1, 0.1]], W=[W, [1, 1, 1]],
                     fixed=[0, 1], K=10)
    s.step(100)
    P = s.particles()
    assert np.allclose(P["X"][0], [11.3, 9.3, 10.2], atol=1e-12)
    assert np.allclose(P["X"][1], [40, 30, 30]) and np.allclose(P["V"][1], 0)
    ang = np.linalg.norm(W) * 100
    axis = W / np.linalg.norm(W)
    q_exact = np.r_[math.cos(ang / 2), math.sin(ang / 2) * axis]
    assert np.allclose(P["q"][0], q_exact, atol=2e-4)


def test_constant_body_force_is_integrated_exactly():
    """Eq. 9 with only F_g: X = X0 + V0 t + F_g t^2 / (2 m) (Verlet is exact)."""
    s, w = _dem_only([[10, 10, 10]], [2.0], V=[[0.01, 0, 0]], K=7)
    w.body_force = (0.0, 0.0, -0.5)
    s = oracle.Oracle(w, lbm_on=False)
    s.step(40)
    m = w.rho_p * 4 / 3 * math.pi * 8
    assert np.allclose(s.particles()["X"][0], [10.4, 10, 10 - 0.5 * 0.5 / m * 1600], atol=1e-11)


def test_oblique_frictional_collisions_conserve_momentum():
    rng = np.random.default_rng(3)
    X = [[20, 20, 20], [29.7, 21.5, 20.5], [20.3, 29.8, 21], [30.5, 31, 19]]
    V = rng.uniform(-0.02, 0.02, (4, 3))
    W = rng.uniform(-0.003, 0.003, (4, 3))
    s, w = _dem_only(X, [5, 5, 5, 5], V=V, W=W, K=10, mu=0.4)
    m = w.rho_p * 4 / 3 * math.pi * 125
    p0 = m * s.particles()["V"].sum(0)
    s.step(150)
    assert np.allclose(m * s.particles()["V"].sum(0), p0, atol=1e-12)


def test_dry_chain_release_wave_speed():
    R, n, d0 = 5.005, 60, 0.01
    X = np.array([[i * (2 * R - d0), 6.0, 6.0] for i in range(1, n + 1)])
    X[0, 0] = 10.001
    w = workloads.Workload(name="chain", nx=620, ny=12, nz=12, tau=1.0, inlet=workloads.X_PERIODIC, X=X,
                           R=np.full(n, R), fixed=np.zeros(n, np.uint8), E_p=10.0, nu_p=0.2, mu=0.0,
                           dem_substeps=10, amplitude=0.0)
    o = oracle.Oracle(w, lbm_on=False)
    o.step(600)
    V = o.particles()["V"]
    o.close()
    m = w.rho_p * 4 / 3 * math.pi * R ** 3
    kn = 2 * w.E_p / (3 * (1 - w.nu_p ** 2))
    v_th = 0.8 * math.sqrt(1.5 * kn * math.sqrt(R / 2) / m) * d0 ** 1.25
    assert abs(-V[5, 0] / v_th - 1) < 5e-3 and abs(V[n - 6, 0] / v_th - 1) < 5e-3
    # the rest of the motion is along the chain
    assert np.abs(V[:, 1:]).max() < 1e-12
