"""lbm_dem_read_particles_noalloc (the sphere read-out that stages its values
in a fixed device array instead of allocating) against lbm_dem_read_particles
through the C ABI, on consecutive calls.  Named to be collected last, so it
also runs after every other GPU test of the session has used the device."""
import numpy as np
import pytest

import workloads
from paper_1808_08921_gb300 import lbmdem

pytestmark = pytest.mark.gpu

KEYS = ("X", "V", "W", "q", "Fh", "Th")


def _same(a, b):
    for k in KEYS:
        scale = max(np.abs(b[k]).max(), 1e-300)
        assert np.abs(a[k] - b[k]).max() <= 1e-12 * scale, k


def test_noalloc_readout_matches_allocating_readout_on_consecutive_calls():
    w = workloads.config_parity(steps=40)
    g = lbmdem.Sim.from_workload(w)
    g.step(3)
    first = g.particles_noalloc()       # the first call on the device sets it up
    _same(first, g.particles())
    again = g.particles_noalloc()        # second call in a row, same state
    _same(again, first)
    g.step(11)                           # the spheres move and feel the fluid
    ref = g.particles()
    second = g.particles_noalloc()
    _same(second, ref)
    assert np.abs(second["X"] - first["X"]).max() > 0   # not the previous contents
    assert np.abs(second["Fh"]).max() > 0
    g.close()


def test_noalloc_readout_rejects_more_spheres_than_its_buffer():
    n = 65537
    side = int(np.ceil(n ** (1 / 3)))
    ijk = np.stack(np.meshgrid(*[np.arange(side)] * 3, indexing="ij"), -1).reshape(-1, 3)[:n]
    X = 2.0 * ijk + 1.0
    w = workloads.Workload(name="many", nx=2 * side, ny=2 * side, nz=2 * side, tau=1.0, X=X,
                           R=np.full(n, 0.4), V=np.zeros((n, 3)), W=np.zeros((n, 3)),
                           fixed=np.zeros(n, np.uint8), dem_substeps=1)
    g = lbmdem.Sim(lbmdem.params_from_workload(w, lbm_on=0, dem_skin=0.5))
    g.set_packing(w.X, w.R, w.V, w.W, w.fixed)
    with pytest.raises(lbmdem.LbmDemError) as e:
        g.particles_noalloc()
    assert "65536" in str(e.value)
    assert g.particles()["X"].shape == (n, 3)     # the allocating read-out still serves it
    g.close()
