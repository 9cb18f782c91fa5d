"""Benchmark of the coupled LBM-DEM step on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload: the 128 x 128 x 1024 column (x = 1024, propagation axis) with 2048
spheres R = 11.4 on an FCC lattice a = 32 (4 x 4 x 32 cells), tau 0.6,
sinusoidal inlet (amplitude 1e-3, period 400), seeded jitter 1e-3 R, FP32
populations; synthetic input from workloads.config_scale().

metric: coupled-step MLUPS over fluid nodes (fluid-node updates per second,
millions), whole job.  `kernel_rooflines` gives, for the HBM-bound kernel
groups, the algorithmic bytes per launch (collide+stream of the odd steps:
152 B per fluid node, 19 FP32 populations read and written; of the even
steps, which take their links inside the same kernel: 152 B plus the node's
8 B link word; the link kernel of the odd steps: 8 B per link record, one
population read and the bounced value written) over the
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
BYTES_PER_LINK_WORD = 8  # per node: the even steps' links inside collide+stream
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


# the sources of the profiled kernels (collide+stream of both parities, the
# link kernel) and the headers they include; host-side launch code is not in it
PROFILED_SOURCES = ("common.cuh", "kernels.cuh", "lattice.cu", "coupling.cu")


def _kernel_hash():
    """Hash of the profiled kernels' source code (comments and layout
    excluded): a profile is valid only for the code it measured."""
    h = hashlib.sha256()
    for name in PROFILED_SOURCES:
        f = os.path.join(ROOT, "paper_1808_08921_gb300", "csrc", name)
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


def make_stream(torch, dev):
    """A dedicated (non-default) CUDA stream for the library and the timing
    events.  The library issues every kernel of a step on the stream it is
    given; handle 0 (torch's legacy default stream) would make it create a
    private stream of its own, which events recorded by the caller never
    wait for -- the events would then time the host enqueue only."""
    s = torch.cuda.Stream(device=dev)
    h = int(s.cuda_stream)
    if h == 0:
        raise RuntimeError("benchmark stream has the default handle 0")
    return s, h


def time_steps(torch, sim, stream, steps, barrier):
    """Device milliseconds of `steps` coupled steps: CUDA events recorded on
    the stream the library launches on, with a barrier and a device
    synchronise on both sides."""
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    barrier()
    return e0.elapsed_time(e1)


def workload_config(w, storage="f32"):
    """The `config` object of both arms (ours and reference): the workload
    by name and its defining sizes, nothing measured."""
    return {"workload": w.name, "lattice": [w.nx, w.ny, w.nz], "spheres": int(w.n_particles),
            "tau": w.tau, "dem_substeps": w.dem_substeps,
            "source": "sine amplitude %g period %g" % (w.amplitude, round(2 * math.pi / w.omega, 3)),
            "population_storage": storage,
            "l2": "no flush: inputs larger than L2 (19 populations per stored node, > 300 MB, "
                  "against 129 MB of L2)"}


def validate(line):
    """Refuse a line whose numbers cannot describe real GPU work: a whole
    step faster than the HBM roofline of its own collide+stream bytes (a
    little above 1.0 is possible against a measured copy peak), or a single
    kernel launch longer than the whole step it belongs to."""
    why = []
    fr = line["step_roofline"]["frac"]
    if fr > 1.2:
        why.append(f"step_roofline.frac {fr} > 1.2")
    us = line["roofline"]["us_per_launch"]
    if us > 1.1 * 1e3 * line["ms_per_step"]:
        why.append(f"dominant kernel {us} us per launch > step {line['ms_per_step']} ms")
    if line["value"] <= 0 or not math.isfinite(line["value"]):
        why.append("non-positive value")
    return why


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
    stream, handle = make_stream(torch, dev)
    storage = {"f32": lbmdem.F32, "bf16": lbmdem.BF16_DEV, "f16": lbmdem.F16_DEV}[args.storage]
    over = dict(device=dev, cuda_stream=handle, skin=0.1, dem_skin=0.5)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    clk = Clocks(dev).__enter__()  # samples from the warm-up to the end of the timed windows
    sim = lbmdem.Sim.from_workload(w, storage=storage, **over)
    sim.step(args.warmup)
    barrier()
    cnt_a = sim.counters()
    ms = time_steps(torch, sim, stream, args.steps, barrier)
    cnt_b = sim.counters()
    # per-kernel-group times over a second window of the same length, with
    # CUDA events recorded around each group inside the captured graphs.
    # Those event nodes cost tens of microseconds per step (they stall the
    # launch pipeline between kernels), so the headline window above runs
    # without them; the group times below include that launch latency.
    sim.set_timing(True)
    ms_timed = time_steps(torch, sim, stream, args.steps, barrier)
    tm = sim.timing()
    sim.set_timing(False)
    st = sim.status()
    fluid = cnt_b["fluid"]
    ms_max, fluid_sum = aggregate(ms, fluid, world, "cuda")
    value = fluid_sum * args.steps / (ms_max * 1e-3) / 1e6
    # rooflines of the HBM-bound kernel groups at their algorithmic bytes
    # (collide+stream: 152 B per fluid node, plus the link word on the even
    # steps when they take their links; links: 8 B per link record, the
    # population read and the bounced value written); the dominant one by
    # measured time is the headline `roofline`
    peak, peak_kind = _peaks()
    esz = 4 if args.storage == "f32" else 2  # bytes per stored population
    node_bytes = BYTES_PER_FLUID_NODE * esz // 4
    fused = tm["links"][1] < tm["collide_odd"][1] + tm["collide_even"][1]
    algo = {"collide_even": (node_bytes + (BYTES_PER_LINK_WORD if fused else 0), fluid, "fluid node"),
            "collide_odd": (node_bytes, fluid, "fluid node"),
            "links": (BYTES_PER_LINK * esz // 4, cnt_b["links"], "link record")}
    kernels = {}
    for g, (per, units, uname) in algo.items():
        k_ms, k_n = tm[g]
        if k_n == 0:
            continue
        avg = k_ms / k_n
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
                     "frac": round(step_ach / peak, 4), "peak_kind": peak_kind,
                     "note": "whole coupled step at the collide+stream bytes per fluid node (all kernels in the time)"}
    launches = cnt_b["launches"] - cnt_a["launches"]
    # the same column with 16-bit population storage, same steps
    storage_runs = {}
    if not args.no_storage and args.storage == "f32" and world == 1:
        for name, code in (("f16", lbmdem.F16_DEV), ("bf16", lbmdem.BF16_DEV)):
            s2 = lbmdem.Sim.from_workload(w, storage=code, **over)
            s2.step(args.warmup)
            m2 = time_steps(torch, s2, stream, args.steps, barrier)
            storage_runs["storage_" + name] = {
                "ms_per_step": round(m2 / args.steps, 4),
                "value": round(s2.counters()["fluid"] * args.steps / (m2 * 1e-3) / 1e6, 1),
                "speedup_vs_f32": round(ms / m2, 3), "status": s2.status(),
                "note": "populations stored as 16-bit deviations f - w rho_f, FP32 arithmetic"}
            s2.close()
        # the precision configuration's own lattice: the 16 x 16 x 128
        # column's physics on a 64 x 64 x 512 crop (2048 spheres R 5.7)
        wc = workloads.config_crop(steps=args.steps)
        crop = {}
        for name, code in (("f32", lbmdem.F32), ("f16", lbmdem.F16_DEV), ("bf16", lbmdem.BF16_DEV)):
            s2 = lbmdem.Sim.from_workload(wc, storage=code, **over)
            s2.step(args.warmup)
            m2 = time_steps(torch, s2, stream, args.steps, barrier)
            crop[name] = {"ms_per_step": round(m2 / args.steps, 4),
                          "value": round(s2.counters()["fluid"] * args.steps / (m2 * 1e-3) / 1e6, 1),
                          "status": s2.status()}
            s2.close()
        for name in ("f16", "bf16"):
            crop[name]["speedup_vs_f32"] = round(crop["f32"]["ms_per_step"] / crop[name]["ms_per_step"], 3)
        storage_runs["storage_crop"] = dict(crop, workload=wc.name, lattice=[wc.nx, wc.ny, wc.nz],
                                            spheres=len(wc.R), unit=UNIT)
    clk.__exit__(None, None, None)
    # end to end through the C ABI from host buffers
    e2e = None
    if not args.no_e2e:
        sim2 = lbmdem.Sim(lbmdem.params_from_workload(w, storage=storage, **over))
        sim2.set_pressure_source(w.waveform, w.amplitude, w.omega, w.t_n, w.t0)
        n = w.n_particles
        h2d = 8 * (3 * n + n + 3 * n + 3 * n) + n  # X, R, V, Omega (FP64) + fixed flags
        d2h = 8 * 19 * n  # X, V, Omega, q, F, T (FP64)
        barrier()
        t0 = time.perf_counter()
        sim2.set_packing(w.X, w.R, np.zeros((n, 3)), np.zeros((n, 3)), w.fixed)
        sim2.step(args.steps)
        sim2.particles()
        barrier()
        t1 = time.perf_counter()
        fl2 = sim2.counters()["fluid"]
        e2e = {"value": round(fl2 * args.steps / (t1 - t0) / 1e6, 1), "unit": UNIT,
               "h2d_bytes_per_step": round(h2d / args.steps, 1),
               "d2h_bytes_per_step": round(d2h / args.steps, 1),
               "includes": "set_packing (host -> device, layout build) + steps + read_particles (device -> host)"}
        sim2.close()
    # the same column with the DEM subcycle the autotuner picks (reported
    # beside the headline, which keeps K = 10)
    tuned = None
    if not args.no_tune and world == 1:
        from paper_1808_08921_gb300 import autotune
        sim.close()
        r = autotune.tune(w, substeps=(1, 2, 3, 5, 10), tiles=(128,), link_modes=(), steps=64,
                          **{k: v for k, v in over.items() if k != "cuda_stream"})
        sim = lbmdem.Sim.from_workload(w, storage=storage, **dict(over, dem_substeps=r["dem_substeps"]))
        sim.step(args.warmup)
        n2 = max(2, args.steps // 2)
        ms2 = time_steps(torch, sim, stream, n2, barrier)
        tuned = {"dem_substeps": r["dem_substeps"], "steps": n2,
                 "value": round(sim.counters()["fluid"] * n2 / (ms2 * 1e-3) / 1e6, 1),
                 "ms_per_step": round(ms2 / n2, 4), "k_table": r["k_table"],
                 "rule": "smallest K whose sphere trajectories over 64 steps stay within 1e-2 of K = 10"}
    adj = None
    if not args.no_adjoint and world == 1:
        with torch.cuda.stream(stream):
            adj = adjoint_record(args.adj_steps, handle)
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
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.storage,
            "data": "synthetic",
            "config": workload_config(w, args.storage),
            "layout": {"fluid_nodes": fluid, "stored_nodes": cnt_b["stored"], "nodes": cnt_b["nodes"],
                       "mlups_all_nodes": round(value * cnt_b["nodes"] / max(fluid, 1), 1),
                       "link_records": cnt_b["links"],
                       "relayouts_in_timed_region": cnt_b["relayouts"] - cnt_a["relayouts"],
                       "conversions_in_timed_region": cnt_b["conversions"] - cnt_a["conversions"],
                       "stream": "dedicated non-default CUDA stream shared by the library and the events",
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
            "adjoint": adj,
        }
        line.update(storage_runs)
        bad = validate(line)
        if bad:
            sys.stderr.write("bench: refusing an impossible measurement: " + "; ".join(bad) + "\n")
            sys.stderr.write(json.dumps(line) + "\n")
            raise SystemExit(3)
        print(json.dumps(line))
    sim.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _oracle_sample(budget_s, threads, o=None):
    """Time the FP64 oracle on the same 128x128x1024 column with `threads`
    OpenMP threads, one step at a time, until the budget is spent (at least
    one step).  Returns (fluid nodes, step times, oracle)."""
    import oracle
    import workloads
    oracle.set_threads(threads)
    if o is None:
        o = oracle.Oracle(workloads.config_scale(steps=1))
    _, _, sol = o.fields()
    fluid = int((sol == 0).sum())
    times = []
    t_start = time.perf_counter()
    while True:
        t0 = time.perf_counter()
        o.step(1)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - t_start > budget_s:
            break
    return fluid, times, o


def cpu_baseline(budget_s):
    """The oracle as it stands (plain FP64 C, OpenMP over x-planes) on the
    host cores: all of them, and one, each for about half the budget."""
    import oracle
    cores = os.cpu_count() or 1
    fluid, t_all, o = _oracle_sample(0.5 * budget_s, cores)
    _, t_one, o = _oracle_sample(0.5 * budget_s, 1, o)
    o.close()
    oracle.set_threads(cores)
    v_all = fluid * len(t_all) / sum(t_all) / 1e6
    v_one = fluid * len(t_one) / sum(t_one) / 1e6
    return {"value": round(v_all, 3), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{len(t_all)} coupled steps of the 128x128x1024 column (2048 spheres), "
                      f"FP64 C with OpenMP over x-planes on {cores} threads, {sum(t_all):.1f} s",
            "single_core": {"value": round(v_one, 3), "unit": UNIT, "cores": 1,
                            "sample": f"{len(t_one)} further steps of the same run on 1 thread, "
                                      f"{sum(t_one):.1f} s"},
            "parallel_speedup": round(v_all / v_one, 2)}


def _slab(cells_x):
    """x-slab of the same FCC column: 128 x 128 cross-section, 32 * cells_x
    lattice units long, same sphere size, spacing, tau and source."""
    import workloads
    return workloads.fcc_column(32 * cells_x, 128, 128, 0.6, 32.0, 11.4, jitter=1e-3 * 11.4,
                                seed=2, period=400, mu=0.3, substeps=10, steps=1,
                                name=f"fcc128x128x{32 * cells_x}_a32_R11.4_tau0.6")


def run_reference(args):
    """The FP64 oracle timed on the host cores (all of them, OpenMP over
    x-planes) on the same workload.  Each step is one coupled oracle step on
    an x-slab of the column (same cross-section and packing), the slab sized
    so that the whole run fits in about args.ref_seconds; MLUPS over fluid
    nodes is comparable across lengths."""
    rank, world, _ = _dist()
    if rank != 0:
        return
    import oracle
    import workloads
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
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
              f"{w.nx}-long x-slab of the 128x128x1024 column ({w.n_particles} spheres, "
              f"{fluid} fluid nodes), FP64 C with OpenMP over x-planes on {cores} threads")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * dt / args.steps, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(workloads.config_scale(steps=args.steps)),
            "cpu_baseline": {"value": round(value, 3), "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_sweep(args):
    """The source sweep: 48 independent columns 32 x 32 x L (L 256..1024, sine
    and Ricker sources, ceil(L sqrt 3) steps each).  The autotuner picks the
    DEM subcycle and the collide+stream tile on the median column; the
    columns then run as one batch (one launch of one CUDA graph: a device-side
    loop per column) and, for comparison, one after another.  value =
    fluid-node updates of all columns per second of the batched run."""
    import torch

    import workloads
    from paper_1808_08921_gb300 import autotune, lbmdem

    ws, steps = workloads.config_sweep(48)
    med = sorted(range(len(ws)), key=lambda k: ws[k].nx)[len(ws) // 2]
    over = dict(skin=0.25, dem_skin=0.5)
    tuned = (autotune.tune(ws[med], steps=96, **over) if not args.no_tune
             else {"dem_substeps": 10, "tile": 256, "link_mode": 0})
    over.update(dem_substeps=tuned["dem_substeps"], tile=tuned["tile"], link_mode=tuned["link_mode"])
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
                       "dem_substeps": over["dem_substeps"], "tile": over["tile"],
                       "link_mode": over["link_mode"]},
            "batch": out["batch"], "sequential": out["sequential"],
            "speedup_vs_sequential": round(out["batch"]["mlups"] / max(out["sequential"]["mlups"], 1e-9), 3),
            "autotune": tuned}
    print(json.dumps(line))


def adjoint_record(steps, stream_handle=None, every=100):
    """Gradient of the probe-plane pressure misfit on the fixed 64 x 64 x 512
    packing (256 spheres R 11.4, probe x = 400, checkpoints every 100): the
    adjoint's cost against the plain forward run, and its gradient against
    central finite differences of the forward loss."""
    import numpy as np

    import workloads
    from paper_1808_08921_gb300 import lbmdem

    w = workloads.config_adjoint(steps)
    tau, amp = w.tau, w.amplitude
    extra = {} if stream_handle is None else {"cuda_stream": stream_handle}

    def sim(t, a):
        s = lbmdem.Sim(lbmdem.params_from_workload(w, tau=t, **extra))
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
    # sphere positions, through the smooth coupling surrogate (outside the
    # paper): its adjoint against its forward run, and dL/dX of the six
    # coordinates of the two spheres nearest the probe against central
    # differences of the surrogate's own loss
    # target: the surrogate's trace at (1.03 tau, 1.2 rho') with seeded noise,
    # so that the residual (and dL/dX) is well above FP32 resolution
    s = sim(1.03 * tau, 1.2 * amp)
    _, ptrace = s.surrogate_loss(steps, np.zeros(steps))
    s.close()
    ptarget = ptrace + np.random.default_rng(8).normal(0.0, 1e-5 / 3.0, steps)
    s = sim(tau, amp)
    s.status()
    t0 = time.perf_counter()
    Lp, _ = s.surrogate_loss(steps, ptarget)
    s.status()
    t_pf = time.perf_counter() - t0
    t0 = time.perf_counter()
    Lp2, dp_tau, dp_amp, dX, _ = s.adjoint_psm(steps, every, ptarget)
    t_pa = time.perf_counter() - t0
    near = np.argsort(np.abs(w.X[:, 0] - w.probe_x))[:2]
    hx = 5e-3
    fd_x, ad_x = [], []
    for p in near:
        for a in range(3):
            Xp, Xm = w.X.copy(), w.X.copy()
            Xp[p, a] += hx
            Xm[p, a] -= hx
            s.set_packing(Xp, w.R, None, None, w.fixed)
            lp, _ = s.surrogate_loss(steps, ptarget)
            s.set_packing(Xm, w.R, None, None, w.fixed)
            lm, _ = s.surrogate_loss(steps, ptarget)
            fd_x.append((lp - lm) / (2 * hx))
            ad_x.append(float(dX[p, a]))
    s.close()
    fd_x, ad_x = np.array(fd_x), np.array(ad_x)
    positions = {"model": "smooth partially-saturated coupling surrogate (outside the paper; lbm_dem_adjoint_psm)",
                 "spheres": len(w.R), "cost_ratio": round(t_pa / t_pf, 3), "forward_s": round(t_pf, 4),
                 "adjoint_s": round(t_pa, 4), "loss": Lp2, "dL_dtau": dp_tau, "dL_damp": dp_amp,
                 "checked": [[int(p), a] for p in near for a in range(3)],
                 "dL_dX_checked": ad_x.tolist(), "fd_dL_dX_checked": fd_x.tolist(),
                 "rel_err_x": float(np.abs(ad_x - fd_x).max() / max(np.abs(fd_x).max(), 1e-300)),
                 "fd_step_lu": hx}
    return {"metric": "adjoint cost / forward cost", "value": round(t_adj / t_fwd, 3), "unit": "ratio",
            "higher_is_better": False,
            "config": {"workload": w.name, "lattice": [w.nx, w.ny, w.nz], "spheres": len(w.R), "steps": steps,
                       "checkpoint_every": every, "probe_x": w.probe_x, "tau": tau, "amplitude": amp},
            "forward_s": round(t_fwd, 4), "adjoint_s": round(t_adj, 4), "loss": L, "loss_forward": L0,
            "dL_dtau": d_tau, "fd_dL_dtau": fd_tau, "rel_err_tau": abs(d_tau - fd_tau) / max(abs(fd_tau), 1e-300),
            "dL_damp": d_amp, "fd_dL_damp": fd_amp, "rel_err_amp": abs(d_amp - fd_amp) / max(abs(fd_amp), 1e-300),
            "positions": positions,
            "timing": "wall clock around a device synchronise on both sides (forward: the steps alone; "
                      "adjoint: forward sweep with checkpoints, recomputation and the reverse sweep)"}


def run_adjoint(args):
    line = adjoint_record(args.adj_steps)
    line.update({"n_gpus": 1, "dtype": "f32", "data": "synthetic"})
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
    ap.add_argument("--no-storage", action="store_true", help="skip the 16-bit storage sub-records")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint sub-record")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=24.0)
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
