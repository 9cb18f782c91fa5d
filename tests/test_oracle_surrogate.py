"""Pins of the oracle's smooth coupling surrogate (for gradients in the sphere
positions; outside the paper's chosen method, which names the Noble-Torczynski
partially-saturated scheme as the alternative family in Section 1).

Every node carries populations and collides with
    f*_i = f_i - (1 - B)/tau (f_i - f^eq_i) + B (f_opp(i) - f_i + w_i rho - f^eq_opp(i)),
    B = eps (tau - 1/2) / ((1 - eps) + (tau - 1/2)),
with eps the smooth solid fraction of the node.  Pinned by:
  * the solid fraction itself: S(R - |x - X| + 1/2) with the cubic
    smoothstep S at chosen distances, the union of two spheres, fluid x ends;
  * eps = 0 reduces the step to the BGK step of the momentum-exchange model
    without spheres;
  * a uniform flow in a periodic box under uniform eps loses the fraction B
    of its momentum per step, exactly ((1 - B)^k): fixes B(eps, tau) and the
    momentum of the solid term;
  * one step is the convex combination (1 - B) step(eps = 0) + B step(eps = 1)
    of a random state; eps = 1 takes an equilibrium to rest at its density;
  * total mass in a closed periodic box with spheres is conserved."""
import math

import numpy as np

import oracle
import workloads


def _box(nx=10, ny=7, nz=6, tau=0.8, X=None, R=None):
    X = np.zeros((0, 3)) if X is None else np.asarray(X, float)
    R = np.zeros(0) if R is None else np.asarray(R, float)
    return workloads.Workload(name="psm", nx=nx, ny=ny, nz=nz, tau=tau, inlet=workloads.X_PERIODIC,
                              X=X, R=R, fixed=np.ones(len(R), np.uint8), dem_substeps=1, amplitude=0.0)


def _psm(w):
    o = oracle.Oracle(w)
    o.set_coupling(True)
    return o


def _smoothstep(v):
    v = min(max(v, 0.0), 1.0)
    return v * v * (3 - 2 * v)


def test_solid_fraction_profile_and_union():
    X = np.array([[6.3, 4.0, 5.0], [6.3, 4.0, 11.2]])
    R = np.array([3.0, 2.6])
    w = _box(nx=14, ny=9, nz=16, X=X, R=R)
    w.inlet, w.outlet = workloads.X_WALL, workloads.OUTLET_WALL
    e = _psm(w).psm_fraction()
    for (x, y, z) in [(6, 4, 5), (9, 4, 5), (3, 4, 5), (6, 4, 8), (8, 6, 5), (5, 2, 3), (6, 4, 14), (6, 4, 9)]:
        keep = 1.0
        for p in range(2):
            d = math.dist((x, y, z), X[p])
            keep *= 1.0 - _smoothstep(R[p] - d + 0.5)
        assert abs(e[x, y, z] - (1.0 - keep)) < 1e-15, (x, y, z)
    assert e[6, 4, 5] == 1.0 and e[6, 4, 11] == 1.0 and e[13, 4, 5] == 0.0
    assert 0.0 < e[6, 4, 8] < 1.0                    # between the spheres: both contribute
    assert (e[0] == 0).all() and (e[-1] == 0).all()  # the x ends stay fluid


def test_zero_fraction_is_the_bgk_step():
    w = _box()
    a, b = oracle.Oracle(w), _psm(w)
    rng = np.random.default_rng(2)
    f = a.populations() * (1 + rng.uniform(-0.02, 0.02, a.populations().shape))
    a.set_populations(f)
    b.set_populations(f)
    a.step(7)
    b.step(7)
    assert np.abs(a.populations() - b.populations()).max() < 1e-15


def test_uniform_fraction_damps_momentum_by_B():
    for eps, tau in [(0.3, 0.6), (0.7, 0.9), (1.0, 0.75), (0.05, 1.4)]:
        w = _box(tau=tau)
        o = _psm(w)
        o.psm_set_fraction(np.full(w.nodes, eps))
        f0 = np.repeat(oracle.equilibrium(1.004, [0.02, -0.013, 0.007])[:, None], w.nodes, 1)
        o.set_populations(f0)
        B = eps * (tau - 0.5) / ((1 - eps) + (tau - 0.5))
        c, _, _ = oracle.lattice()
        j0 = np.einsum("mn,ma->a", f0, c)
        for k in range(1, 5):
            o.step(1)
            f = o.populations().reshape(19, -1)
            j = np.einsum("mn,ma->a", f, c)
            assert np.abs(j - (1 - B) ** k * j0).max() < 1e-12 * np.abs(j0).max() + 1e-15, (eps, tau, k)
            assert abs(f.sum() - f0.sum()) < 1e-12 * f0.sum()


def test_step_is_convex_combination_and_full_solid_rests():
    eps, tau = 0.42, 0.7
    B = eps * (tau - 0.5) / ((1 - eps) + (tau - 0.5))
    w = _box(tau=tau)
    rng = np.random.default_rng(5)
    base = oracle.Oracle(w).populations()
    f = base * (1 + rng.uniform(-0.03, 0.03, base.shape))
    out = []
    for e in (eps, 0.0, 1.0):
        o = _psm(w)
        o.psm_set_fraction(np.full(w.nodes, e))
        o.set_populations(f)
        o.step(1)
        out.append(o.populations())
    assert np.abs(out[0] - ((1 - B) * out[1] + B * out[2])).max() < 1e-15
    o = _psm(w)
    o.psm_set_fraction(np.ones(w.nodes))
    feq = oracle.equilibrium(1.01, [0.03, 0.01, -0.02])
    o.set_populations(np.repeat(feq[:, None], w.nodes, 1))
    o.step(1)
    _, wts, _ = oracle.lattice()
    assert np.abs(o.populations().reshape(19, -1) - (wts * 1.01)[:, None]).max() < 1e-15


def test_closed_box_with_spheres_conserves_mass():
    w = _box(nx=16, ny=12, nz=12, X=[[5.2, 6.1, 5.7], [11.4, 3.3, 8.8]], R=[3.1, 2.7])
    o = _psm(w)
    rng = np.random.default_rng(8)
    f = o.populations() * (1 + rng.uniform(-0.01, 0.01, o.populations().shape))
    o.set_populations(f)
    m0 = f.sum()
    o.step(40)
    assert abs(o.populations().sum() - m0) < 1e-12 * m0
