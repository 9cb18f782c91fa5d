"""Device-side failure reporting without a GPU fault: a run driven unstable
(tau near 1/2, a large source) latches LBMDEM_ERR_UNSTABLE in the status
word, every later call reports it, and the context is still released
cleanly; a healthy context on the same device is unaffected."""
import numpy as np
import pytest

import workloads
from paper_1808_08921_gb300 import lbmdem

pytestmark = pytest.mark.gpu


def test_unstable_run_is_reported_and_latched():
    w = workloads.plane_wave(nx=64, ny=2, nz=2, tau=0.5001, amplitude=1.5, omega=0.5, steps=400)
    g = lbmdem.Sim.from_workload(w, monitor_every=1)
    with pytest.raises(lbmdem.LbmDemError) as e:
        for _ in range(50):
            g.step(16)
            g.status()
    assert e.value.code == -4  # LBMDEM_ERR_UNSTABLE
    with pytest.raises(lbmdem.LbmDemError):
        g.step(2)
    g.close()
    ok = lbmdem.Sim.from_workload(workloads.plane_wave(nx=64, ny=2, nz=2, steps=10))
    ok.step(10)
    assert ok.status() == 0
    rho, _, _ = ok.fields()
    assert np.isfinite(rho).all()
    ok.close()
