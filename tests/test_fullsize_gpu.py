"""GPU parity at full size: the 128x128x1024 column (2048 spheres R 11.4 on
FCC a = 32, tau 0.6) in the configuration the benchmark times -- FP32
populations, steps captured in one 16-step CUDA graph, re-layout skin 0.1,
DEM neighbour skin 0.5, 64-thread collide+stream blocks, 10 DEM substeps --
against the FP64 oracle on the same seeded input, over every node and every
sphere (the oracle takes ~1.5 s per step here, so 16 steps).

The column starts at rest with seeded sphere velocities of up to 2e-3 lu per
step, so that after one graph the flow reaches every pore, spheres collide
through their initial overlaps, and band nodes are covered and uncovered
(the conversions of Eqs. 16-17) all along the column; the inlet wave enters
at x = 0.  Bars as in test_parity_gpu.
"""
import numpy as np
import pytest

import oracle
import workloads
from paper_1808_08921_gb300 import lbmdem
from test_parity_gpu import compare_fields, compare_particles

pytestmark = pytest.mark.gpu


def test_full_size_column_in_the_benchmark_configuration():
    w = workloads.config_scale(steps=16)
    n = w.n_particles
    rng = np.random.default_rng(1808)
    mobile = (w.fixed == 0)[:, None]
    w.V = np.where(mobile, rng.uniform(-2e-3, 2e-3, (n, 3)), 0.0)
    w.W = np.where(mobile, rng.uniform(-2e-4, 2e-4, (n, 3)), 0.0)
    g = lbmdem.Sim.from_workload(w, skin=0.1, dem_skin=0.5, tile=64, graph_steps=16)
    o = oracle.Oracle(w)
    g.step(16)
    o.step(16)
    c = g.counters()
    assert c["conversions"] > 0, "the seeded motion should cover and uncover band nodes"
    assert c["relayouts"] == 0
    dr, du, sig, umax = compare_fields(g, o)
    dx = compare_particles(g, o)
    print(f"full size, 16 steps: |drho| {dr:.3e} (signal {sig:.3e}), |du| {du:.3e} (max {umax:.3e}), "
          f"|dX| {dx:.3e}, conversions {c['conversions']}")
    g.close()
    o.close()
