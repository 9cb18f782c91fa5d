"""The seeded input generators (CPU): the workloads have the geometry the
input recipe states -- FCC centres a(i, j, k) + a b + a/4 with the 4-point
basis, end layers along x fixed and unperturbed, seeded jitter within its
half-width, the sphere counts and overlaps of each configuration, and the
source sweep's lengths and periods -- and the same seed gives the same input."""
import math

import numpy as np
import pytest

import workloads


def _min_pair_distance(X, box):
    d = X[:, None, :] - X[None, :, :]
    for a, L in enumerate(box):
        if L:
            d[..., a] -= L * np.round(d[..., a] / L)
    r = np.sqrt((d * d).sum(-1))
    np.fill_diagonal(r, np.inf)
    return r.min()


def test_fcc_unit_cell_positions():
    X, R, fixed = workloads.fcc_packing(4.0, (1, 1, 1), 1.0, fix_end_layers=False)
    expect = 4.0 * np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]]) + 1.0
    assert np.array_equal(X, expect)
    assert np.array_equal(R, np.ones(4)) and not fixed.any()


@pytest.mark.parametrize("make,n,nx,R,a", [
    (workloads.config_parity, 32, 128, 5.7, 16.0),
    (workloads.config_scale, 2048, 1024, 11.4, 32.0),
    (workloads.config_crop, 2048, 512, 5.7, 16.0),
    (workloads.config_adjoint, 256, 512, 11.4, 32.0),
])
def test_column_geometry(make, n, nx, R, a):
    w = make(steps=1)
    assert w.n_particles == n and w.nx == nx and np.all(w.R == R)
    assert np.all((w.X[:, 0] > 0) & (w.X[:, 0] < w.nx))
    assert np.all((w.X[:, 1:] >= 0) & (w.X[:, 1:] < [w.ny, w.nz]))
    # nearest neighbours at a / sqrt(2) (up to the jitter), periodic in y, z
    dmin = _min_pair_distance(w.X, (0, w.ny, w.nz))
    assert abs(dmin - a / math.sqrt(2)) < 0.1


def test_scale_column_overlap_and_fixed_layers():
    w = workloads.config_scale(steps=1)
    # R = 11.4 on a = 32 taken literally: neighbours overlap by 2R - a/sqrt(2)
    assert abs((2 * 11.4 - 32 / math.sqrt(2)) - 0.1726) < 1e-3
    xs = np.sort(np.unique(np.round(w.X[w.fixed == 1, 0], 6)))
    X0, _, _ = workloads.fcc_packing(32.0, (32, 4, 4), 11.4, jitter=0.0)
    layers = np.sort(np.unique(np.round(X0[:, 0], 6)))
    assert np.array_equal(xs, layers[[0, -1]])  # lowest and highest x layer
    assert w.fixed.sum() == 2 * 32  # 4 x 4 cells x 2 basis points per x layer
    # fixed spheres are exactly on the lattice, free ones within the jitter
    d = np.abs(w.X - X0)
    assert d[w.fixed == 1].max() == 0.0
    assert 0 < d[w.fixed == 0].max() <= 1e-3 * 11.4


def test_seed_reproducibility():
    a, b = workloads.config_scale(steps=1), workloads.config_scale(steps=1)
    assert np.array_equal(a.X, b.X)
    c = workloads.fcc_column(1024, 128, 128, 0.6, 32.0, 11.4, jitter=1e-3 * 11.4, seed=3, period=400)
    assert not np.array_equal(a.X, c.X)


def test_sweep_lengths_and_periods():
    ws, steps = workloads.config_sweep()
    assert len(ws) == 48
    L = np.array([w.nx for w in ws])
    assert np.all(L % 16 == 0) and L.min() >= 256 and L.max() <= 1024
    assert all(w.ny == 32 and w.nz == 32 for w in ws)
    assert steps == [math.ceil(l * math.sqrt(3)) for l in L]
    sines = [w for w in ws if w.waveform == workloads.SINE]
    rickers = [w for w in ws if w.waveform == workloads.RICKER]
    assert len(sines) == 40 and len(rickers) == 8
    periods = np.array([2 * math.pi / w.omega for w in sines])
    assert abs(periods.min() - 50) < 1e-9 and abs(periods.max() - 800) < 1e-9
    assert np.allclose(np.diff(np.log(periods)), np.log(16) / 39)  # log-spaced
