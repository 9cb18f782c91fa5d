"""An even step's links taken inside its collide+stream kernel (link_mode 2,
the default for FP32 storage and spheres of radius 8 lu or more: link words
per node, sphere sums per warp) against the link
kernel every step (link_mode 1), and both against the FP64 oracle, including
a fluid node whose solid neighbours belong to three spheres (the link word's
owner-map fallback).

The two modes evaluate the same Eqs. 14-15 and 18-19 with different FP32
operation orders (the wall velocity at the node against per-direction
moving-wall terms; per-warp sums in another order), so they agree to FP32
rounding, far inside the oracle bars of test_parity_gpu.
"""
import math

import numpy as np
import pytest

import oracle
import workloads
from paper_1808_08921_gb300 import lbmdem
from test_parity_gpu import compare_fields, compare_particles

pytestmark = pytest.mark.gpu


def _run(w, steps, mode, **over):
    s = lbmdem.Sim.from_workload(w, link_mode=mode, **over)
    try:
        s.step(steps)
        return s.fields(), s.particles(), s.counters(), s.status()
    finally:
        s.close()


def _close(a, b, R, bars=(2e-6, 2e-5, 1e-6, 2e-5)):
    """The two link paths against each other.  bars: density as a fraction of
    the density signal, velocity of max |u|, centres in lu, force and torque
    of their largest component; the default is FP32 summation order."""
    br, bu, bx, bf = bars
    (rg, ug, sg), pa, ca, sta = a
    (ro, uo, so), pb, cb, stb = b
    assert sta == 0 and stb == 0
    assert np.array_equal(sg, so)
    fl = so == 0
    assert np.abs(rg - ro)[fl].max() <= br * max(np.abs(ro[fl] - 1.0).max(), 1e-6)
    assert np.abs(ug - uo).max() <= bu * np.abs(uo).max() + 1e-12
    if len(pa["X"]):
        assert np.abs(pa["X"] - pb["X"]).max() <= bx
        fs = np.abs(pb["Fh"]).max()
        assert np.abs(pa["Fh"] - pb["Fh"]).max() <= bf * fs + 1e-12
        ts = max(np.abs(pb["Th"]).max(), R * fs)
        assert np.abs(pa["Th"] - pb["Th"]).max() <= bf * ts + 1e-12
    assert ca["conversions"] == cb["conversions"]


@pytest.mark.parametrize("steps", [1, 2, 41])
def test_links_in_collide_match_the_link_kernel(steps):
    """Moving spheres with conversions, after an even last step (1, 41) and an
    odd one (2)."""
    w = workloads.random_small(5, nx=40, ny=20, nz=20, n=8, R=3.5, vel=0.02, steps=steps)
    _close(_run(w, steps, 2), _run(w, steps, 1), 3.5)


def _three_spheres():
    """Three fixed spheres overlapping pairwise around the x axis line
    (y, z) = (10, 10): the node there is fluid and has solid neighbours of
    all three."""
    R, side = 3.0, 5.7
    d = side / math.sqrt(3.0)
    X = np.array([[10.0, 10.0 + d * math.cos(a), 10.0 + d * math.sin(a)]
                  for a in (math.pi / 2, math.pi / 2 + 2 * math.pi / 3, math.pi / 2 + 4 * math.pi / 3)])
    return workloads.Workload(name="three", nx=20, ny=20, nz=20, tau=0.8, X=X, R=np.full(3, R),
                              fixed=np.ones(3, np.uint8), amplitude=2e-3, omega=2 * math.pi / 40,
                              dem_substeps=2)


def test_three_sphere_node_exists():
    w = _three_spheres()
    o = oracle.Oracle(w)
    own = o.owner()
    c, _, _ = oracle.lattice()
    found = 0
    for x in range(1, w.nx - 1):
        for y in range(w.ny):
            for z in range(w.nz):
                if own[x, y, z] >= 0:
                    continue
                ps = {own[x + c[m, 0], (y + c[m, 1]) % w.ny, (z + c[m, 2]) % w.nz] for m in range(18)}
                ps.discard(-1)
                found += len([p for p in ps if p >= 0]) >= 3
    assert found > 0


@pytest.mark.parametrize("steps", [1, 30])
def test_three_sphere_links_match_oracle_and_link_kernel(steps):
    w = _three_spheres()
    a, b = _run(w, steps, 2), _run(w, steps, 1)
    _close(a, b, 3.0)
    o = oracle.Oracle(w)
    o.step(steps)
    g = lbmdem.Sim.from_workload(w, link_mode=2)
    try:
        g.step(steps)
        compare_fields(g, o)
        compare_particles(g, o, R=w.R)
    finally:
        g.close()


def _launches(w, steps, mode, **over):
    s = lbmdem.Sim.from_workload(w, link_mode=mode, **over)
    try:
        s.step(steps)
        return s.counters()["launches"]
    finally:
        s.close()


def test_narrow_periodic_box_keeps_the_link_lists():
    """Where a node can neighbour two periodic images of one sphere (the
    12 x 12 cross-section of the saturated chains, R = 5.005) every step uses
    the link lists, whose records carry the lever of their own image, even
    when the collide kernel's links are asked for; a wide box takes the even
    steps' links in the collide kernel with link_mode 2 (one launch fewer per
    even step), and by default only with spheres of radius 8 lu or more."""
    narrow = workloads.saturated_chain(True, steps=4)
    assert _launches(narrow, 4, 0) == _launches(narrow, 4, 1) == _launches(narrow, 4, 2)
    wide = workloads.random_small(5, nx=40, ny=20, nz=20, n=8, R=3.5, vel=0.02, steps=4)
    assert _launches(wide, 4, 1) - _launches(wide, 4, 2) == 2
    assert _launches(wide, 4, 0) == _launches(wide, 4, 1)
    large = workloads.random_small(6, nx=48, ny=28, nz=28, n=2, R=8.5, vel=0.02, steps=4)
    assert _launches(large, 4, 1) - _launches(large, 4, 0) == 2
    # the default takes the link kernel with 16-bit storage; mode 2 forces the
    # collide kernel's links there too
    assert _launches(large, 4, 0, storage=lbmdem.F16_DEV) == _launches(large, 4, 1, storage=lbmdem.F16_DEV)
    f16 = dict(storage=lbmdem.F16_DEV)
    assert _launches(wide, 4, 0, **f16) == _launches(wide, 4, 1, **f16)
    assert _launches(wide, 4, 1, **f16) - _launches(wide, 4, 2, **f16) == 2


# 16-bit storage rounds the two paths' slightly different FP32 values to
# different 16-bit neighbours now and then, so the paths differ by the
# storage's own rounding noise: the field bars of test_storage_gpu (density
# of the signal, velocity of max |u|), ten times its centre bars (these
# light R = 3.5 spheres move with the link sums' 16-bit noise within 21
# steps: measured 1.6e-6 lu FP16, 1.0e-5 lu BF16) and ten times the density
# bar for the link sums
BARS16 = {"F16_DEV": (2e-3, 1e-1, 1e-5, 2e-2), "BF16_DEV": (2e-2, 5e-1, 1e-4, 2e-1)}


@pytest.mark.parametrize("storage", ["F16_DEV", "BF16_DEV"])
def test_links_in_collide_with_16_bit_storage(storage):
    """The collide kernel's links on 16-bit populations (link_mode 2) against
    the link kernel on the same storage."""
    w = workloads.random_small(5, nx=40, ny=20, nz=20, n=8, R=3.5, vel=0.02, steps=21)
    st = dict(storage=getattr(lbmdem, storage))
    _close(_run(w, 21, 2, **st), _run(w, 21, 1, **st), 3.5, BARS16[storage])
