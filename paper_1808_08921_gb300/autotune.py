"""Autotuner for columns of the source sweep: the DEM subcycle K, the
collide+stream block size ("tile") and the link path (link_mode: the even
steps' links inside the collide kernel, or the link kernel every step),
measured on scratch copies of a column.

K sets the DEM time step 1/K of a coupled step (Section 2.2: the spheres
move with the fluid's time step, subdivided for the contact stiffness).  The
tuner runs the column with the largest candidate K as reference and keeps
the smallest K whose sphere trajectories stay within `tol` of it (relative to
the largest displacement of the reference run) with a clean device status;
then it times every tile at that K and keeps the fastest, then both link
paths at that K and tile (they give the same results up to FP32 summation
order) and keeps the faster.  Scratch runs use the column's own workload;
the caller's simulation is not touched.
"""
from __future__ import annotations

import time

import numpy as np

from . import lbmdem


def _run(w, steps, **over):
    s = lbmdem.Sim.from_workload(w, **over)
    x0 = s.particles()["X"].copy()
    s.step(steps)
    st = s.status()
    x1 = s.particles()["X"]
    s.close()
    return x0, x1, st


def _time(w, steps, warm, **over):
    s = lbmdem.Sim.from_workload(w, **over)
    s.step(warm)
    s.status()
    t0 = time.perf_counter()
    s.step(steps)
    st = s.status()
    dt = time.perf_counter() - t0
    s.close()
    return dt / steps, st


def tune(w, substeps=(2, 3, 4, 5, 6, 8, 10, 16), tiles=(64, 128, 256), link_modes=(2, 1), steps=128, tol=1e-2,
         warm=32, **over):
    """Returns {"dem_substeps": K, "tile": T, "link_mode": M, "k_table": [...],
    "tile_table": [...], "link_table": [...]}; a link_mode given in `over` is
    kept rather than tuned."""
    ks = sorted(set(int(k) for k in substeps))
    x0, xref, st = _run(w, steps, dem_substeps=ks[-1], **over)
    if st != 0:
        raise lbmdem.LbmDemError(st, f"reference run with K = {ks[-1]} failed")
    scale = max(float(np.abs(xref - x0).max()), 1e-12)
    k_table, best_k = [], ks[-1]
    for k in ks[:-1]:
        _, x1, st = _run(w, steps, dem_substeps=k, **over)
        err = float(np.abs(x1 - xref).max()) / scale if st == 0 else float("inf")
        k_table.append({"dem_substeps": k, "rel_err": err, "status": st})
        if st == 0 and err <= tol and k < best_k:
            best_k = k
            break  # candidates ascend: the first that passes is the smallest
    k_table.append({"dem_substeps": ks[-1], "rel_err": 0.0, "status": 0})
    tile_table = []
    for t in tiles:
        sec, st = _time(w, steps, warm, dem_substeps=best_k, tile=int(t), **over)
        tile_table.append({"tile": int(t), "us_per_step": 1e6 * sec, "status": st})
    ok = [r for r in tile_table if r["status"] == 0]
    best_t = min(ok, key=lambda r: r["us_per_step"])["tile"] if ok else 256
    link_table = []
    if "link_mode" in over:
        best_m = int(over["link_mode"])
    else:
        for mdx in link_modes:
            sec, st = _time(w, steps, warm, dem_substeps=best_k, tile=best_t, link_mode=int(mdx), **over)
            link_table.append({"link_mode": int(mdx), "us_per_step": 1e6 * sec, "status": st})
        okm = [r for r in link_table if r["status"] == 0]
        best_m = min(okm, key=lambda r: r["us_per_step"])["link_mode"] if okm else 0
    return {"dem_substeps": best_k, "tile": best_t, "link_mode": best_m, "k_table": k_table,
            "tile_table": tile_table, "link_table": link_table}
