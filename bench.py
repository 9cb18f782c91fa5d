"""Benchmark of the coupled LBM-DEM step on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload: the 128 x 128 x 1024 column (x = 1024, propagation axis) with 2048
spheres R = 11.4 on an FCC lattice a = 32 (4 x 4 x 32 cells), tau 0.6,
sinusoidal inlet (amplitude 1e-3, period 400), seeded jitter 1e-3 R, FP32
populations; synthetic input from workloads.config_scale().

metric: coupled-step MLUPS over fluid nodes (fluid-node updates per second,
millions), whole job.  `kernel_rooflines` gives, for the HBM-bound kernel
groups, the algorithmic bytes per launch (collide+stream, both AA parities:
152 B per fluid node, 19 FP32 populations read and written; links: 8 B per
link record, one population read and the bounced value written) over the
group's mean launch time, taken with CUDA events around every launch inside
the captured graphs during a second window of K steps that follows the
headline window (those event nodes slow the step, so the headline `value`
is timed without them); `roofline` is the one with the longest launches,
and `step_roofline` is the whole coupled step at 152 B per fluid node.
`e2e` times the same workload through the C ABI from host buffers:
set_packing (host -> device, the layout build included), the K steps, and
the read-back of the sphere state (device -> host).  `cpu_baseline` times
the FP64 oracle on a few steps of the same workload on the host cores.  Multi-GPU (torchrun): every rank runs its
own column (independent problems, no collective), value = all ranks' fluid
updates / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES_PER_FLUID_NODE = 152  # 19 populations x 4 B, read + write
BYTES_PER_LINK = 8  # one population read, the bounced value written
METRIC = "coupled step MLUPS (fluid nodes)"
UNIT = "MLUPS"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        import tempfile
        self.path = os.path.join(tempfile.gettempdir(), f"lbmdem_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5], f[6], f[7], f[8]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[2 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def _code_only(text):
    """C/CUDA source without comments and whitespace (the sources hold no
    string literal with a comment marker)."""
    import re
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return re.sub(r"\s+", "", text)


def _kernel_hash():
    """Hash of the CUDA sources' code (comments and layout excluded): a
    profile is valid only for the code it measured."""
    import glob
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(ROOT, "paper_1808_08921_gb300", "csrc", "*.cu*"))):
        h.update(_code_only(open(f).read()).encode())
    return h.hexdigest()[:16]


PROFILE = os.path.join(ROOT, "profiles", "coupled_step_fcc128x128x1024.md")


def _profiled_traffic(group):
    """DRAM bytes per launch of a kernel group from the committed ncu summary,
    if it was taken on the current kernel sources (else None)."""
    if not os.path.exists(PROFILE):
        return None
    kh, val = None, None
    key = f"dram_bytes_per_launch[{group}]:"
    for line in open(PROFILE).read().splitlines():
        if line.startswith("kernel_source_hash:"):
            kh = line.split(":", 1)[1].strip()
        if line.startswith(key):
            try:
                val = float(line.split(":", 1)[1].strip())
            except ValueError:
                val = None
    return val if kh == _kernel_hash() else None


def aggregate(ms, fluid, world, device):
    """Whole-job figures of a multi-rank run (independent columns, one per
    rank): the slowest rank's time and all ranks' fluid nodes.  The only
    collective of the benchmark; the step itself exchanges nothing."""
    if world <= 1:
        return ms, float(fluid)
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms, float(fluid)], device=device, dtype=torch.float64)
    ts = [torch.zeros_like(t) for _ in range(world)]
    dist.all_gather(ts, t)
    return max(float(x[0]) for x in ts), sum(float(x[1]) for x in ts)


def run_ours(args):
    import numpy as np
    import torch

    import workloads
    from paper_1808_08921_gb300 import lbmdem

    rank, world, local = _dist()
    dev = local
    torch.cuda.set_device(dev)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", dev))
    w = workloads.config_scale(steps=args.steps)
    stream = torch.cuda.current_stream()
    storage = {"f32": lbmdem.F32, "bf16": lbmdem.BF16_DEV, "f16": lbmdem.F16_DEV}[args.storage]
    over = dict(device=dev, cuda_stream=stream.cuda_stream, skin=0.1, dem_skin=0.5, storage=storage)
    sim = lbmdem.Sim.from_workload(w, **over)
    cnt0 = sim.counters()
    sim.step(args.warmup)
    torch.cuda.synchronize()
    cnt_a = sim.counters()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    barrier()
    with Clocks(dev) as clk:
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        sim.step(args.steps)
        ev1.record(stream)
        barrier()
    ms = ev0.elapsed_time(ev1)
    cnt_b = sim.counters()
    # per-kernel-group times over a second window of the same length, with
    # CUDA events recorded around each group inside the captured graphs.
    # Those event nodes cost tens of microseconds per step (they stall the
    # launch pipeline between kernels), so the headline window above runs
    # without them; the group times below include that launch latency.
    sim.set_timing(True)
    barrier()
    ev2 = torch.cuda.Event(enable_timing=True)
    ev3 = torch.cuda.Event(enable_timing=True)
    ev2.record(stream)
    sim.step(args.steps)
    ev3.record(stream)
    barrier()
    ms_timed = ev2.elapsed_time(ev3)
    tm = sim.timing()
    sim.set_timing(False)
    st = sim.status()
    fluid = cnt_b["fluid"]
    ms_max, fluid_sum = aggregate(ms, fluid, world, "cuda")
    value = fluid_sum * args.steps / (ms_max * 1e-3) / 1e6
    # rooflines of the HBM-bound kernel groups at their algorithmic bytes
    # (collide+stream: 152 B per fluid node; links: 8 B per link record, the
    # population read and the bounced value written); the dominant one by
    # measured time is the headline `roofline`
    peak, peak_kind = _peaks()
    esz = 4 if args.storage == "f32" else 2  # bytes per stored population
    node_bytes = BYTES_PER_FLUID_NODE * esz // 4
    algo = {"collide_stream": (node_bytes, fluid, "fluid node"),
            "links": (BYTES_PER_LINK * esz // 4, cnt_b["links"], "link record")}
    kernels = {}
    for g, (per, units, uname) in algo.items():
        k_ms, k_n = tm[g]
        avg = k_ms / max(k_n, 1)
        ach = per * units / (avg * 1e-3) / 1e9 if avg > 0 else 0.0
        kernels[g] = {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                      "frac": round(ach / peak, 4), "traffic": _profiled_traffic(g),
                      "bytes_per_launch": per * units, "bytes_per_unit": per, "units": units,
                      "work_unit": uname, "us_per_launch": round(1e3 * avg, 2), "peak_kind": peak_kind}
    dom = max(kernels, key=lambda g: kernels[g]["us_per_launch"])
    roofline = dict(kernels[dom], kernel=dom)
    step_bytes = node_bytes * fluid_sum
    step_ach = step_bytes * args.steps / (ms_max * 1e-3) / 1e9
    step_roofline = {"bytes_per_step": step_bytes, "achieved": round(step_ach, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(step_ach / peak, 4),
                     "note": "whole coupled step at the collide+stream bytes per fluid node (all kernels in the time)"}
    # end to end through the C ABI from host buffers
    e2e = None
    if not args.no_e2e:
        sim2 = lbmdem.Sim(lbmdem.params_from_workload(w, **over))
        sim2.set_pressure_source(w.waveform, w.amplitude, w.omega, w.t_n, w.t0)
        n = w.n_particles
        h2d = 8 * (3 * n + n + 3 * n + 3 * n) + n  # X, R, V, Omega (FP64) + fixed flags
        d2h = 8 * 19 * n  # X, V, Omega, q, F, T (FP64)
        barrier()
        t0 = time.perf_counter()
        sim2.set_packing(w.X, w.R, np.zeros((n, 3)), np.zeros((n, 3)), w.fixed)
        sim2.step(args.steps)
        P = sim2.particles()
        barrier()
        t1 = time.perf_counter()
        fl2 = sim2.counters()["fluid"]
        e2e = {"value": round(fl2 * args.steps / (t1 - t0) / 1e6, 1), "unit": UNIT,
               "h2d_bytes_per_step": round(h2d / args.steps, 1),
               "d2h_bytes_per_step": round(d2h / args.steps, 1),
               "includes": "set_packing (layout build) + steps + read_particles"}
        sim2.close()
    launches = cnt_b["launches"] - cnt_a["launches"]
    # the same column with the DEM subcycle the autotuner picks (reported
    # beside the headline, which keeps K = 10)
    tuned = None
    if not args.no_tune and world == 1:
        from paper_1808_08921_gb300 import autotune
        sim.close()
        r = autotune.tune(w, substeps=(1, 2, 3, 5, 10), tiles=(128,), steps=64, **{k: v for k, v in over.items()
                                                                                    if k != "cuda_stream"})
        sim = lbmdem.Sim.from_workload(w, **dict(over, dem_substeps=r["dem_substeps"]))
        sim.step(args.warmup)
        n2 = max(2, args.steps // 2)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        sim.step(n2)
        e1.record(stream)
        torch.cuda.synchronize()
        ms2 = e0.elapsed_time(e1)
        tuned = {"dem_substeps": r["dem_substeps"], "steps": n2,
                 "value": round(sim.counters()["fluid"] * n2 / (ms2 * 1e-3) / 1e6, 1),
                 "ms_per_step": round(ms2 / n2, 4), "k_table": r["k_table"],
                 "rule": "smallest K whose sphere trajectories over 64 steps stay within 1e-2 of K = 10"}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(args.cpu_seconds)
    if rank == 0:
        groups = {k: {"ms_total": round(v[0], 3), "launches": v[1],
                      "us_avg": round(1e3 * v[0] / max(v[1], 1), 2)} for k, v in tm.items()}
        groups["window"] = {"steps": args.steps, "ms_per_step_with_events": round(ms_timed / args.steps, 4),
                            "note": "second window after the headline one; CUDA events around each "
                                    "kernel group inside the graphs"}
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": w.name, "lattice": [w.nx, w.ny, w.nz], "spheres": w.n_particles,
                       "fluid_nodes": fluid, "stored_nodes": cnt_b["stored"], "tau": w.tau,
                       "dem_substeps": w.dem_substeps, "source": "sine amplitude 1e-3 period 400",
                       "mlups_all_nodes": round(value * cnt_b["nodes"] / max(fluid, 1), 1),
                       "l2": "inputs larger than L2: populations %.0f MB" % (19 * 4 * cnt_b["stored"] / 1e6),
                       "relayouts_in_timed_region": cnt_b["relayouts"] - cnt_a["relayouts"],
                       "conversions_in_timed_region": cnt_b["conversions"] - cnt_a["conversions"],
                       "link_records": cnt_b["links"],
                       "population_storage": args.storage,
                       "status": st},
            "roofline": roofline,
            "step_roofline": step_roofline,
            "kernel_rooflines": kernels,
            "kernel_groups": groups,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
            "autotuned_dem_substeps": tuned,
        }
        print(json.dumps(line))
    sim.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _oracle_sample(steps_budget_s, max_steps=None):
    """Time the FP64 oracle on the same 128x128x1024 column, one step at a
    time, until the budget is spent (at least one step)."""
    import oracle
    import workloads
    w = workloads.config_scale(steps=1)
    o = oracle.Oracle(w)
    _, _, sol = o.fields()
    fluid = int((sol == 0).sum())
    times = []
    t_start = time.perf_counter()
    while True:
        t0 = time.perf_counter()
        o.step(1)
        times.append(time.perf_counter() - t0)
        if max_steps and len(times) >= max_steps:
            break
        if not max_steps and time.perf_counter() - t_start > steps_budget_s:
            break
    o.close()
    return fluid, times


def cpu_baseline(budget_s):
    fluid, times = _oracle_sample(budget_s)
    mlups = fluid * len(times) / sum(times) / 1e6
    return {"value": round(mlups, 3), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{len(times)} coupled steps of the 128x128x1024 column (2048 spheres), "
                      f"FP64 single-threaded C, {sum(times):.1f} s"}


def _slab(cells_x):
    """x-slab of the same FCC column: 128 x 128 cross-section, 32 * cells_x
    lattice units long, same sphere size, spacing, tau and source."""
    import workloads
    return workloads.fcc_column(32 * cells_x, 128, 128, 0.6, 32.0, 11.4, jitter=1e-3 * 11.4,
                                seed=2, period=400, mu=0.3, substeps=10, steps=1,
                                name=f"fcc128x128x{32 * cells_x}_a32_R11.4_tau0.6")


def run_reference(args):
    """The FP64 oracle timed on the host cores on the same workload.  Each
    step is one coupled oracle step on an x-slab of the column (same cross-
    section and packing), the slab sized so that the whole run fits in about
    args.ref_seconds; MLUPS over fluid nodes is comparable across lengths."""
    rank, world, _ = _dist()
    if rank != 0:
        return
    import oracle
    w1 = _slab(1)
    o = oracle.Oracle(w1)
    t0 = time.perf_counter()
    o.step(1)
    t1 = time.perf_counter() - t0
    o.close()
    per_step = args.ref_seconds / max(args.steps + args.warmup, 1)
    cells = int(max(1, min(32, per_step / max(t1, 1e-6))))
    w = _slab(cells)
    o = oracle.Oracle(w)
    _, _, sol = o.fields()
    fluid = int((sol == 0).sum())
    for _ in range(args.warmup):
        o.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(1)
    dt = time.perf_counter() - t0
    o.close()
    value = fluid * args.steps / dt / 1e6
    sample = (f"{args.steps} timed coupled steps (+{args.warmup} warm-up) of a "
              f"{w.nx}-long x-slab of the 128x128x1024 column ({w.n_particles} spheres), "
              f"FP64 single-threaded C")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * dt / args.steps, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "fcc128x128x1024_a32_R11.4_tau0.6", "sample_lattice": [w.nx, w.ny, w.nz],
                       "sample_spheres": w.n_particles, "sample_fluid_nodes": fluid},
            "cpu_baseline": {"value": round(value, 3), "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_sweep(args):
    """The source sweep: 48 independent columns 32 x 32 x L (L 256..1024, sine
    and Ricker sources, ceil(L sqrt 3) steps each).  The autotuner picks the
    DEM subcycle and the collide+stream tile on the median column; the
    columns then run as one batch (one CUDA graph per 16-step chunk) and, for
    comparison, one after another.  value = fluid-node updates of all columns
    per second of the batched run."""
    import torch

    import workloads
    from paper_1808_08921_gb300 import autotune, lbmdem

    ws, steps = workloads.config_sweep(48)
    med = sorted(range(len(ws)), key=lambda k: ws[k].nx)[len(ws) // 2]
    over = dict(skin=0.25, dem_skin=0.5)
    tuned = autotune.tune(ws[med], steps=96, **over) if not args.no_tune else {"dem_substeps": 10, "tile": 256}
    over.update(dem_substeps=tuned["dem_substeps"], tile=tuned["tile"])
    out = {}
    for mode in ("batch", "sequential"):
        sims = [lbmdem.Sim.from_workload(w, **over) for w in ws]
        fluid = [s.counters()["fluid"] for s in sims]
        torch.cuda.synchronize()
        with Clocks(0) as clk:
            t0 = time.perf_counter()
            if mode == "batch":
                b = lbmdem.Batch(sims)
                b.step(steps)
                b.sync()
                gl = b.graph_launches
                b.close()
            else:
                for s, k in zip(sims, steps):
                    s.step(k)
                for s in sims:
                    s.status()
                gl = 0
            dt = time.perf_counter() - t0
        st = max(abs(s.status()) for s in sims)
        upd = sum(f * k for f, k in zip(fluid, steps))
        out[mode] = {"s": round(dt, 3), "mlups": round(upd / dt / 1e6, 1), "graph_launches": gl, "status": st,
                     "clocks": clk.summary()}
        for s in sims:
            s.close()
    line = {"metric": "source sweep MLUPS (fluid nodes, 48 columns)", "value": out["batch"]["mlups"], "unit": UNIT,
            "n_gpus": 1, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "sweep48_32x32xL_a16_R5.7_tau0.8", "columns": len(ws),
                       "lengths": [w.nx for w in ws], "steps": steps, "fluid_updates": upd,
                       "dem_substeps": over["dem_substeps"], "tile": over["tile"]},
            "batch": out["batch"], "sequential": out["sequential"],
            "speedup_vs_sequential": round(out["batch"]["mlups"] / max(out["sequential"]["mlups"], 1e-9), 3),
            "autotune": tuned}
    print(json.dumps(line))


def run_adjoint(args):
    """Gradient of the probe-plane pressure misfit on the fixed 64 x 64 x 512
    packing (256 spheres R 11.4, probe x = 400, 5000 steps, checkpoints every
    100): the adjoint's cost against the plain forward run, and its gradient
    against central finite differences of the forward loss."""
    import numpy as np

    import workloads
    from paper_1808_08921_gb300 import adjoint, lbmdem

    steps, every = args.adj_steps, 100
    w = workloads.config_adjoint(steps)
    tau, amp = w.tau, w.amplitude

    def sim(t, a):
        s = lbmdem.Sim(lbmdem.params_from_workload(w, tau=t))
        s.set_pressure_source(w.waveform, a, w.omega, w.t_n, w.t0)
        s.set_packing(w.X, w.R, None, None, w.fixed)
        return s

    # target: the forward trace at (tau, amp) with a seeded N(0, 1e-5 rho_f c_s^2) perturbation
    s = sim(tau, amp)
    s.step(steps)
    base = s.probe()[:steps] / 3.0
    s.close()
    target = base + np.random.default_rng(7).normal(0.0, 1e-5 / 3.0, steps)

    def forward_loss(t, a):
        s = sim(t, a)
        s.status()
        t0 = time.perf_counter()
        s.step(steps)
        s.status()
        dt = time.perf_counter() - t0
        p = s.probe()[:steps] / 3.0
        s.close()
        return float(((p - target) ** 2).sum()), dt

    L0, t_fwd = forward_loss(tau, amp)
    s = sim(tau, amp)
    s.status()
    t0 = time.perf_counter()
    L, d_tau, d_amp, _ = s.adjoint(steps, every, target)
    t_adj = time.perf_counter() - t0
    s.close()
    h, ha = 1e-3 * tau, 1e-2 * amp
    fd_tau = (forward_loss(tau + h, amp)[0] - forward_loss(tau - h, amp)[0]) / (2 * h)
    fd_amp = (forward_loss(tau, amp + ha)[0] - forward_loss(tau, amp - ha)[0]) / (2 * ha)
    line = {"metric": "adjoint cost / forward cost", "value": round(t_adj / t_fwd, 3), "unit": "ratio",
            "higher_is_better": False, "n_gpus": 1, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "lattice": [w.nx, w.ny, w.nz], "spheres": len(w.R), "steps": steps,
                       "checkpoint_every": every, "probe_x": w.probe_x, "tau": tau, "amplitude": amp},
            "forward_s": round(t_fwd, 4), "adjoint_s": round(t_adj, 4), "loss": L, "loss_forward": L0,
            "dL_dtau": d_tau, "fd_dL_dtau": fd_tau, "rel_err_tau": abs(d_tau - fd_tau) / max(abs(fd_tau), 1e-300),
            "dL_damp": d_amp, "fd_dL_damp": fd_amp, "rel_err_amp": abs(d_amp - fd_amp) / max(abs(fd_amp), 1e-300)}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=None)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--storage", default="f32", choices=["f32", "bf16", "f16"],
                    help="population storage (deviations; the arithmetic is FP32 in every case)")
    ap.add_argument("--sweep", action="store_true",
                    help="the 48-column source sweep (batched, autotuned) instead of the single column")
    ap.add_argument("--no-tune", action="store_true", help="sweep without the autotuner (K = 10, tile 256)")
    ap.add_argument("--adjoint", action="store_true",
                    help="the adjoint's cost and gradient check on the fixed 64 x 64 x 512 packing")
    ap.add_argument("--adj-steps", type=int, default=5000)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-seconds", type=float, default=150.0)
    args = ap.parse_args()
    if args.impl == "reference":
        args.steps = 20 if args.steps is None else args.steps
        args.warmup = 3 if args.warmup is None else args.warmup
        run_reference(args)
        return
    if args.sweep:
        run_sweep(args)
        return
    if args.adjoint:
        run_adjoint(args)
        return
    args.steps = 2000 if args.steps is None else args.steps
    args.warmup = 200 if args.warmup is None else args.warmup
    if args.warmup < 3:
        args.warmup = 3
    run_ours(args)


if __name__ == "__main__":
    main()
