"""Error of the stored populations' precision on the 64 x 64 x 512 crop (the
16 x 16 x 128 column's physics with 2048 spheres) after 2000 coupled steps,
against samples of the FP64 oracle's state written by
tests/golden/make_crop_reference.py: density and velocity on three planes,
the probe trace, and every sphere's centre.  Prints the errors for FP32,
BF16 and FP16 storage; the bars are those of the 16 x 16 x 128 storage test.
"""
import os

import numpy as np
import pytest

import workloads
from paper_1808_08921_gb300 import lbmdem

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "crop64x64x512_oracle.npz")
BARS = {lbmdem.F32: (1e-3, 1e-4, 1e-6),
        lbmdem.F16_DEV: (2e-3, 1e-1, 1e-6),
        lbmdem.BF16_DEV: (2e-2, 5e-1, 1e-5)}


@pytest.mark.parametrize("storage", [lbmdem.F32, lbmdem.F16_DEV, lbmdem.BF16_DEV])
def test_crop_storage_error(storage):
    if not os.path.exists(GOLDEN):
        pytest.skip("oracle samples not generated: run tests/golden/make_crop_reference.py")
    ref = np.load(GOLDEN)
    steps, planes = int(ref["steps"]), list(ref["planes"])
    w = workloads.config_crop(steps=steps)
    w.probe_x = int(ref["probe_x"])
    g = lbmdem.Sim.from_workload(w, storage=storage)
    g.step(steps)
    rho, u, sol = g.fields()
    assert np.array_equal(sol[planes], ref["solid"]), "solid maps differ"
    fl = ref["solid"] == 0
    sig = np.abs(ref["rho"][fl] - 1.0).max()
    drho = np.abs(rho[planes] - ref["rho"])[fl].max() / sig
    du = np.abs(u[:, planes] - ref["u"]).max() / np.abs(ref["u"]).max()
    P = g.particles()
    dx = np.abs(P["X"] - ref["X"]).max()
    pr = g.probe()
    dp = np.abs(pr - ref["probe"]).max() / np.abs(ref["probe"] - 1.0).max()
    print(f"crop storage {storage}: |drho|/rho' {drho:.2e}  |du|/umax {du:.2e}  |dX| {dx:.2e} lu  "
          f"probe {dp:.2e}")
    br, bu, bx = BARS[storage]
    assert drho <= br and du <= bu and dx <= bx and dp <= br, (drho, du, dx, dp)
    g.close()
