"""Write tests/golden/crop64x64x512_oracle.npz: samples of the FP64 oracle's
state after the coupled run of the 64 x 64 x 512 crop (the 16 x 16 x 128
column's physics, tau 0.8, 2048 spheres R 5.7 on FCC a = 16, seed 3), used to
state the error of the GPU path's FP32 and 16-bit population storage.

    python tests/golden/make_crop_reference.py [--steps 2000]

Calls only the oracle (single-threaded FP64 C; about an hour of CPU time for
2000 steps).  Stored: the density and velocity on the planes x = 64, 256 and
448, the solid map there, the probe trace at x = 256, and the sphere centres,
velocities and hydrodynamic forces.
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads  # noqa: E402

PLANES = (64, 256, 448)
PROBE_X = 256


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--out", default=os.path.join(HERE, "crop64x64x512_oracle.npz"))
    a = ap.parse_args()
    w = workloads.config_crop(steps=a.steps)
    w.probe_x = PROBE_X
    o = oracle.Oracle(w)
    t0 = time.time()
    done = 0
    while done < a.steps:
        n = min(100, a.steps - done)
        o.step(n)
        done += n
        print(f"{done} steps, {time.time() - t0:.0f} s", flush=True)
    rho, u, sol = o.fields()
    P = o.particles()
    np.savez_compressed(
        a.out, steps=np.int64(a.steps), planes=np.array(PLANES), probe_x=np.int64(PROBE_X),
        rho=rho[list(PLANES)], u=u[:, list(PLANES)], solid=sol[list(PLANES)], probe=o.probe(),
        X=P["X"], V=P["V"], Fh=P["Fh"])
    print("wrote", a.out)


if __name__ == "__main__":
    main()
