"""Seeded synthetic workloads for the coupled LBM-DEM step.

This module only *generates inputs*: sphere packings, lattice sizes and
source settings.  It holds none of the method's arithmetic, so both the
FP64 oracle (tests) and the CUDA library (tests, bench) may use it.

Geometry conventions (shared by both sides):
  * the lattice is indexed [x][y][z], z fastest; x is the propagation axis
    (inlet at x = 0, outlet at x = nx - 1), y and z are periodic;
  * sphere centres are given in lattice units in the same (x, y, z) frame.

Packings follow the paper's FCC media (Section 4.1): equal spheres on a
face-centred-cubic lattice of cell size ``a``, with the first and last
layers along x fixed in space (Section 4.1, fixed boundary layers).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Waveform ids (Eq. 25 and Table 2 of the paper, plus a Ricker pulse).
SINE, COSINE, STEP, RICKER = 0, 1, 2, 3
# x-boundary modes.
INLET_PRESSURE, X_WALL, X_PERIODIC = 0, 1, 2
OUTLET_ZERO_GRADIENT, OUTLET_PRESSURE, OUTLET_WALL = 0, 1, 2

# Contact-law and solid constants of Table 1 (dimensionless column).
E_P, NU_P, RHO_P = 10.37, 0.2, 2.466


def fcc_packing(a: float, cells: tuple[int, int, int], R: float, *,
                jitter: float = 0.0, seed: int = 1, origin: float | None = None,
                fix_end_layers: bool = True):
    """FCC centres a*(i,j,k) + a*b + origin, b in the 4-point basis.

    Returns (X[n,3], R[n], fixed[n] uint8).  ``jitter`` is the half-width of
    a seeded uniform perturbation applied to every coordinate of every free
    sphere.  Fixed spheres (lowest and highest x layer) are not jittered.
    """
    if origin is None:
        origin = a / 4.0
    basis = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0],
                      [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])
    pts = []
    for i in range(cells[0]):
        for j in range(cells[1]):
            for k in range(cells[2]):
                for b in basis:
                    pts.append(a * (np.array([i, j, k], float) + b) + origin)
    X = np.array(pts, dtype=np.float64)
    n = X.shape[0]
    fixed = np.zeros(n, np.uint8)
    if fix_end_layers:
        xs = X[:, 0]
        fixed[np.isclose(xs, xs.min())] = 1
        fixed[np.isclose(xs, xs.max())] = 1
    if jitter > 0:
        rng = np.random.default_rng(seed)
        d = rng.uniform(-jitter, jitter, size=X.shape)
        d[fixed == 1] = 0.0
        X = X + d
    Rs = np.full(n, float(R))
    return X, Rs, fixed


@dataclass
class Workload:
    """Lattice, physics and packing of one synthetic case."""
    name: str
    nx: int
    ny: int
    nz: int
    tau: float
    rho_f: float = 1.0
    inlet: int = INLET_PRESSURE
    outlet: int = OUTLET_ZERO_GRADIENT
    dem_substeps: int = 10
    E_p: float = E_P
    nu_p: float = NU_P
    mu: float = 0.3
    rho_p: float = RHO_P
    body_force: tuple = (0.0, 0.0, 0.0)
    probe_x: int = -1
    waveform: int = SINE
    amplitude: float = 1e-3
    omega: float = 2 * math.pi / 200
    t_n: int = -1
    t0: float = 0.0
    steps: int = 100
    X: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    R: np.ndarray = field(default_factory=lambda: np.zeros(0))
    fixed: np.ndarray = field(default_factory=lambda: np.zeros(0, np.uint8))
    V: np.ndarray | None = None
    W: np.ndarray | None = None

    @property
    def nodes(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n_particles(self) -> int:
        return int(self.X.shape[0])


def fcc_column(nx, ny, nz, tau, a, R, *, jitter, seed, period, amplitude=1e-3,
               mu=0.3, substeps=10, steps=100, name="fcc", **kw) -> Workload:
    """Column nx x ny x nz filled with FCC cells of size a (cells = dims / a)."""
    cells = (int(round(nx / a)), int(round(ny / a)), int(round(nz / a)))
    X, Rs, fixed = fcc_packing(a, cells, R, jitter=jitter, seed=seed)
    return Workload(name=name, nx=nx, ny=ny, nz=nz, tau=tau, mu=mu,
                    dem_substeps=substeps, amplitude=amplitude,
                    omega=2 * math.pi / period, steps=steps,
                    X=X, R=Rs, fixed=fixed, **kw)


def config_parity(steps: int = 2000) -> Workload:
    """16x16x128 column, tau 0.8, 32 spheres R 5.7 on FCC a = 16, jitter
    +-0.01, sine inlet rho = 1 + 1e-3 sin(2 pi t / 200), zero-gradient outlet,
    mu 0.3, 10 DEM substeps per LBM step."""
    return fcc_column(128, 16, 16, 0.8, 16.0, 5.7, jitter=0.01, seed=1,
                      period=200, mu=0.3, substeps=10, steps=steps,
                      name="fcc16x16x128_a16_R5.7_tau0.8")


def config_scale(steps: int = 20000) -> Workload:
    """128x128x1024 column, tau 0.6, 2048 spheres R 11.4 on FCC a = 32
    (4x4x32 cells), seeded jitter +-1e-3 R, sine period 400, amplitude 1e-3."""
    return fcc_column(1024, 128, 128, 0.6, 32.0, 11.4, jitter=1e-3 * 11.4,
                      seed=2, period=400, mu=0.3, substeps=10, steps=steps,
                      name="fcc128x128x1024_a32_R11.4_tau0.6")


def config_crop(steps: int = 2000) -> Workload:
    """Physics of the 16x16x128 case on a 64x64x512 lattice (2048 spheres)."""
    return fcc_column(512, 64, 64, 0.8, 16.0, 5.7, jitter=0.01, seed=3,
                      period=200, mu=0.3, substeps=10, steps=steps,
                      name="fcc64x64x512_a16_R5.7_tau0.8")


def plane_wave(nx=620, ny=2, nz=2, tau=1.0, amplitude=1e-4, omega=0.03,
               t_n=5000, steps=800) -> Workload:
    """Pure-fluid plane wave of Section 3.2 (source at x = 0, pressure
    locked to rho_f at the far end); the cross-section is uniform, so a
    thin periodic cross-section carries the same 1D solution."""
    return Workload(name=f"wave{ny}x{nz}x{nx}", nx=nx, ny=ny, nz=nz, tau=tau,
                    outlet=OUTLET_PRESSURE, amplitude=amplitude, omega=omega,
                    t_n=t_n, steps=steps, dem_substeps=1)


def saturated_chain(mobile: bool, steps: int = 800, n: int = 60, R: float = 5.005, overlap: float = 0.01,
                    dem_substeps: int = 10) -> Workload:
    """Saturated granular chain of Section 3.2 (third and fourth benchmark):
    the 12 x 12 x 620 fluid domain of the plane wave (tau 1, source rho' 1e-4
    with omega 0.03 at x = 0 for t_n = 5000 steps, pressure locked to rho_f at
    the far end), with 60 spheres of radius 5.005 at x = i (2R - 0.01),
    i = 1..60, on the axis y = z = 6, overlapping by 0.01 at every contact;
    Hertz normal contacts with E = 10, nu = 0.2 and no friction.  The paper
    gives no particle density for the chain: the Table's rho_p is used.
    mobile: every sphere free but the first and the last, which are held
    (third benchmark; reading: the paper calls the equal overlaps of the
    chain its rest state, disturbed only by the source or by shifting the
    first sphere, which a chain with free ends is not: it would release its
    precompression from both ends); else every sphere fixed (fourth
    benchmark)."""
    X = np.array([[i * (2 * R - overlap), 6.0, 6.0] for i in range(1, n + 1)])
    fixed = np.zeros(n, np.uint8) if mobile else np.ones(n, np.uint8)
    fixed[0] = fixed[-1] = 1
    return Workload(name=f"chain{'_mobile' if mobile else '_fixed'}_12x12x620", nx=620, ny=12, nz=12,
                    tau=1.0, outlet=OUTLET_PRESSURE, amplitude=1e-4, omega=0.03, t_n=5000, steps=steps,
                    E_p=10.0, nu_p=0.2, mu=0.0, dem_substeps=dem_substeps, X=X, R=np.full(n, R), fixed=fixed)


def random_small(seed: int, nx=20, ny=12, nz=12, n=4, R=2.5, tau=0.7,
                 mobile=True, vel=0.0, steps=40) -> Workload:
    """A few non-overlapping spheres at random places in a small column,
    used for per-feature parity cases (ragged sizes, several links per node)."""
    rng = np.random.default_rng(seed)
    X = []
    tries = 0
    while len(X) < n and tries < 10000:
        tries += 1
        p = np.array([rng.uniform(R + 2, nx - R - 2), rng.uniform(0, ny),
                      rng.uniform(0, nz)])
        ok = True
        for q in X:
            d = p - q
            d[1] -= ny * round(d[1] / ny)
            d[2] -= nz * round(d[2] / nz)
            if np.linalg.norm(d) < 2 * R + 0.5:
                ok = False
                break
        if ok:
            X.append(p)
    X = np.array(X)
    m = X.shape[0]
    V = rng.uniform(-vel, vel, size=(m, 3)) if vel > 0 else None
    W = rng.uniform(-vel / R, vel / R, size=(m, 3)) if vel > 0 else None
    fixed = np.zeros(m, np.uint8) if mobile else np.ones(m, np.uint8)
    return Workload(name=f"rand{seed}", nx=nx, ny=ny, nz=nz, tau=tau, X=X,
                    R=np.full(m, R), fixed=fixed, V=V, W=W, steps=steps,
                    dem_substeps=4)


def config_sweep(n: int = 48, seed: int = 4, amplitude: float = 1e-3):
    """Source sweep of independent columns: cross-section 32 x 32, lengths
    drawn uniformly from the multiples of 16 in [256, 1024], FCC a = 16 with
    R = 5.7 (the 16 x 16 x 128 column's physics, tau 0.8).  The first
    n - n // 6 columns carry sine sources with periods log-spaced from 50 to
    800 steps, the rest Ricker pulses over the same periods.  Each column
    runs until its front reaches the outlet, ceil(L sqrt(3)) steps.

    Returns (workloads, steps)."""
    rng = np.random.default_rng(seed)
    lengths = 16 * rng.integers(16, 65, size=n)
    n_ricker = n // 6
    n_sine = n - n_ricker
    periods = list(np.geomspace(50, 800, n_sine)) + list(np.geomspace(50, 800, max(n_ricker, 1)))[:n_ricker]
    ws, steps = [], []
    for k in range(n):
        L = int(lengths[k])
        w = fcc_column(L, 32, 32, 0.8, 16.0, 5.7, jitter=0.01, seed=seed * 1000 + k,
                       period=float(periods[k]), amplitude=amplitude, mu=0.3, substeps=10,
                       name=f"sweep{k}_32x32x{L}")
        if k >= n_sine:
            w.waveform = RICKER
            w.t0 = float(periods[k])  # one period of the peak frequency
        ws.append(w)
        steps.append(int(math.ceil(L * math.sqrt(3.0))))
    return ws, steps


def config_adjoint(steps: int = 5000) -> Workload:
    """Fixed packing for the adjoint: 64 x 64 x 512 (x = 512), tau 0.6, FCC
    a = 32 with R = 11.4 (2 x 2 x 16 cells, 256 spheres, every one fixed),
    sine source amplitude 1e-3 with period 400, probe plane x = 400."""
    w = fcc_column(512, 64, 64, 0.6, 32.0, 11.4, jitter=1e-3 * 11.4, seed=5, period=400, mu=0.3,
                   substeps=1, steps=steps, name="fcc64x64x512_a32_R11.4_fixed")
    w.fixed = np.ones(len(w.R), np.uint8)
    w.probe_x = 400
    return w
