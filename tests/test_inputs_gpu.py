"""Failure injection on the host: corrupted packings handed to
lbm_dem_set_packing come back as LBMDEM_ERR_INVALID_ARG with a message, the
context keeps its previous state and accepts a valid packing afterwards, and
stepping before any packing is refused.  No GPU fault is involved."""
import numpy as np
import pytest

import workloads
from paper_1808_08921_gb300 import lbmdem

pytestmark = pytest.mark.gpu

INVALID_ARG = -1


def _good():
    return workloads.random_small(3, nx=30, ny=16, nz=16, n=4, R=3.0, tau=0.8, mobile=True, vel=0.01, steps=8)


def _corrupt(kind, w):
    X, R = w.X.copy(), w.R.copy()
    if kind == "nan_x":
        X[1, 2] = np.nan
    elif kind == "inf_x":
        X[0, 0] = np.inf
    elif kind == "zero_radius":
        R[2] = 0.0
    elif kind == "negative_radius":
        R[0] = -1.0
    elif kind == "deep_overlap":  # two centres closer than the smaller radius
        X[1] = X[0] + np.array([0.0, 0.5, 0.0])
    elif kind == "radius_beyond_half_box":  # R + skin >= L / 2 on the periodic axes
        R[:] = 8.5
    return X, R


@pytest.mark.parametrize("kind", ["nan_x", "inf_x", "zero_radius", "negative_radius", "deep_overlap",
                                  "radius_beyond_half_box"])
def test_corrupt_packing_is_refused_and_the_context_stays_usable(kind):
    w = _good()
    s = lbmdem.Sim(lbmdem.params_from_workload(w))
    try:
        s.set_pressure_source(w.waveform, w.amplitude, w.omega, w.t_n, w.t0)
        X, R = _corrupt(kind, w)
        with pytest.raises(lbmdem.LbmDemError) as e:
            s.set_packing(X, R, w.V, w.W, w.fixed)
        assert e.value.code == INVALID_ARG
        # no packing yet: stepping is refused, not run on stale state
        with pytest.raises(lbmdem.LbmDemError):
            s.step(1)
        s.set_packing(w.X, w.R, w.V, w.W, w.fixed)
        s.step(8)
        assert s.status() == 0
        rho, _, _ = s.fields()
        assert np.isfinite(rho).all()
    finally:
        s.close()
