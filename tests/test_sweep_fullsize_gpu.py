"""GPU parity of the batched source sweep at full size: all 48 columns of the
sweep (32 x 32 x L, L from 256 to 1024, sine and Ricker sources) advanced
together as one batch in the configuration the sweep benchmark times
(re-layout skin 0.25, DEM skin 0.5, the DEM subcycle K = 2 and 64-thread
collide+stream blocks its autotuner picks), 32 steps; the longest column and
a Ricker column against the FP64 oracle with the same K, over every node and
sphere (bars as in test_parity_gpu)."""
import numpy as np
import pytest

import oracle
import workloads
from paper_1808_08921_gb300 import lbmdem
from test_parity_gpu import compare_fields, compare_particles

pytestmark = pytest.mark.gpu

K, TILE, STEPS = 2, 64, 32


def test_full_sweep_batch_against_oracle():
    ws, _ = workloads.config_sweep()
    for w in ws:
        w.dem_substeps = K
    over = dict(skin=0.25, dem_skin=0.5, tile=TILE)
    sims = [lbmdem.Sim.from_workload(w, **over) for w in ws]
    b = lbmdem.Batch(sims)
    b.step([STEPS] * len(ws))
    b.sync()
    assert max(abs(s.status()) for s in sims) == 0
    longest = max(range(len(ws)), key=lambda k: ws[k].nx)
    ricker = next(k for k, w in enumerate(ws) if w.waveform == workloads.RICKER)
    for k in (longest, ricker):
        o = oracle.Oracle(ws[k])
        o.step(STEPS)
        dr, du, sig, umax = compare_fields(sims[k], o)
        dx = compare_particles(sims[k], o)
        print(f"sweep column {k} (32x32x{ws[k].nx}): |drho| {dr:.3e} (signal {sig:.3e}), "
              f"|du| {du:.3e} (max {umax:.3e}), |dX| {dx:.3e}")
        o.close()
    b.close()
    for s in sims:
        s.close()
