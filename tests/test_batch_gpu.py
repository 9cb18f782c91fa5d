"""Batched columns (lbm_dem_batch_*) through the C ABI: several independent
columns of different lengths, sources and step counts advanced together, in
one graph launch per call, give the same state as each column advanced
alone; one batched column stays in parity with the FP64 oracle; the batch's
time limit stops the device loops with LBMDEM_ERR_TIMEOUT (no fault, other
contexts unaffected)."""
import numpy as np
import pytest

import oracle
import workloads
from paper_1808_08921_gb300 import lbmdem

pytestmark = pytest.mark.gpu


def _columns():
    ws = []
    for k, (L, period, wf) in enumerate([(64, 60.0, workloads.SINE), (96, 120.0, workloads.RICKER),
                                          (128, 200.0, workloads.SINE)]):
        w = workloads.fcc_column(L, 32, 32, 0.8, 16.0, 5.7, jitter=0.01, seed=50 + k, period=period,
                                 amplitude=1e-3, substeps=10, name=f"col{k}")
        w.waveform = wf
        w.t0 = period
        w.probe_x = L // 2
        ws.append(w)
    return ws


def test_batch_matches_columns_run_alone():
    ws = _columns()
    steps = [53, 70, 35]  # uneven, odd: chunks, leftovers and parity alignment
    alone = [lbmdem.Sim.from_workload(w) for w in ws]
    for s, n in zip(alone, steps):
        s.step(n)
    cols = [lbmdem.Sim.from_workload(w) for w in ws]
    b = lbmdem.Batch(cols)
    b.step(steps[:2] + [0])
    b.step([0, 0, steps[2]])
    b.sync()
    assert b.graph_launches == 2  # one launch per call, whatever the counts
    for s, g, n in zip(alone, cols, steps):
        r0, u0, s0 = s.fields()
        r1, u1, s1 = g.fields()
        assert np.array_equal(s0, s1)
        fl = s0 == 0
        sig = np.abs(r0[fl] - 1.0).max()
        assert np.abs(r1 - r0)[fl].max() <= 1e-6 * sig
        assert np.abs(u1 - u0).max() <= 1e-6 * np.abs(u0).max()
        p0, p1 = s.particles(), g.particles()
        assert np.abs(p1["X"] - p0["X"]).max() <= 1e-9
        assert np.array_equal(s.probe(), g.probe()) or np.abs(s.probe() - g.probe()).max() <= 1e-9
        assert g.counters()["t"] == n
    b.close()


def test_batched_column_parity_with_oracle():
    w = _columns()[1]
    g = lbmdem.Sim.from_workload(w)
    other = lbmdem.Sim.from_workload(_columns()[0])
    b = lbmdem.Batch([g, other])
    b.step([48, 32])
    b.sync()
    o = oracle.Oracle(w)
    o.step(48)
    rg, ug, sg = g.fields()
    ro, uo, so = o.fields()
    assert np.array_equal(sg, so)
    fl = so == 0
    assert np.abs(rg - ro)[fl].max() <= 1e-3 * np.abs(ro[fl] - 1.0).max()
    assert np.abs(ug - uo).max() <= 1e-4 * np.abs(uo).max()
    assert np.abs(g.particles()["X"] - o.particles()["X"]).max() <= 1e-6
    b.close()


def test_batch_rejects_bad_arguments():
    ws = _columns()
    s = lbmdem.Sim.from_workload(ws[0])
    with pytest.raises(lbmdem.LbmDemError):
        lbmdem.Batch([s, s])
    b = lbmdem.Batch([s])
    with pytest.raises(lbmdem.LbmDemError):
        b.step([-1])
    b.close()


def test_one_launch_runs_uneven_columns_to_completion():
    """Odd and even counts, one of them zero, all in a single graph launch."""
    ws = _columns()
    steps = [41, 0, 64]
    cols = [lbmdem.Sim.from_workload(w) for w in ws]
    alone = [lbmdem.Sim.from_workload(w) for w in ws]
    b = lbmdem.Batch(cols)
    b.step(steps)
    b.sync()
    assert b.graph_launches == 1
    for g, s, n in zip(cols, alone, steps):
        s.step(n)
        assert g.counters()["t"] == n
        assert np.abs(g.particles()["X"] - s.particles()["X"]).max() <= 1e-9
        r0, _, s0 = s.fields()
        r1, _, s1 = g.fields()
        assert np.array_equal(s0, s1) and np.abs(r1 - r0)[s0 == 0].max() <= 1e-9
    b.close()


def test_time_limit_stops_the_loops_with_timeout():
    """A limit far shorter than the run: every column's device loop stops
    between steps and latches LBMDEM_ERR_TIMEOUT; the columns stay readable at
    the step they reached, and a context outside the batch is unaffected."""
    ws = _columns()
    cols = [lbmdem.Sim.from_workload(w) for w in ws]
    b = lbmdem.Batch(cols)
    b.set_time_limit(1e-6)
    b.step([400, 400, 400])
    with pytest.raises(lbmdem.LbmDemError) as ei:
        b.sync()
    assert ei.value.code == -5  # LBMDEM_ERR_TIMEOUT
    import ctypes as C
    for g in cols:
        assert g.status() == -5
        t = g.counters()["t"]
        assert 2 <= t < 400 and t % 2 == 0
        # the state stays readable; the read reports the latched status
        r, u = np.zeros(g.N), np.zeros(3 * g.N)
        rc = lbmdem.load().lbm_dem_read_fields(g._h, r.ctypes.data_as(C.POINTER(C.c_double)),
                                               u.ctypes.data_as(C.POINTER(C.c_double)), None)
        assert rc == -5
        assert np.isfinite(r).all() and np.isfinite(u).all() and r.max() > 0.9
    other = lbmdem.Sim.from_workload(ws[0])
    other.step(20)
    assert other.status() == 0
    b.close()
