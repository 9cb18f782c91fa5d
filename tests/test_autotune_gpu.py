"""The sweep autotuner picks the smallest DEM subcycle within tolerance of
the reference subcycle, the fastest collide+stream tile and the faster link
path, on scratch runs, and a tiled run stays in parity with the oracle."""
import numpy as np
import pytest

import oracle
import workloads
from paper_1808_08921_gb300 import autotune, lbmdem

pytestmark = pytest.mark.gpu


def _column():
    return workloads.fcc_column(128, 32, 32, 0.8, 16.0, 5.7, jitter=0.01, seed=9, period=100.0,
                                amplitude=1e-3, substeps=10, name="tune")


def test_tune_column():
    r = autotune.tune(_column(), substeps=(2, 5, 10, 20), tiles=(64, 128, 256), steps=64, tol=1e-2)
    assert r["dem_substeps"] in (2, 5, 10, 20)
    assert r["tile"] in (64, 128, 256)
    chosen = [row for row in r["k_table"] if row["dem_substeps"] == r["dem_substeps"]][0]
    assert chosen["status"] == 0 and chosen["rel_err"] <= 1e-2
    assert len(r["tile_table"]) == 3 and all(t["status"] == 0 for t in r["tile_table"])
    assert r["link_mode"] in (1, 2)
    assert len(r["link_table"]) == 2 and all(t["status"] == 0 for t in r["link_table"])
    fastest = min(r["link_table"], key=lambda t: t["us_per_step"])
    assert fastest["link_mode"] == r["link_mode"]


@pytest.mark.parametrize("tile", [64, 128])
def test_tile_keeps_parity(tile):
    w = workloads.config_parity(steps=40)
    g = lbmdem.Sim.from_workload(w, tile=tile)
    o = oracle.Oracle(w)
    g.step(40)
    o.step(40)
    rg, ug, sg = g.fields()
    ro, uo, so = o.fields()
    assert np.array_equal(sg, so)
    fl = so == 0
    assert np.abs(rg - ro)[fl].max() <= 1e-3 * np.abs(ro[fl] - 1.0).max()
    assert np.abs(ug - uo).max() <= 1e-4 * np.abs(uo).max()


def test_bad_tile_rejected():
    w = workloads.config_parity(steps=1)
    with pytest.raises(lbmdem.LbmDemError):
        lbmdem.Sim(lbmdem.params_from_workload(w, tile=96))
