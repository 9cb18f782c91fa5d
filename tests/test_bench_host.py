"""Host logic of the benchmark (CPU only): the committed profile summary is
taken as the DRAM traffic of a kernel group only while the CUDA code it
measured is unchanged -- comment and layout edits keep it valid, any code
edit invalidates it."""
import os
import shutil
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_code_only_ignores_comments_and_layout():
    a = "int f(int x) {  // one\n    return x + 1; /* two\n lines */\n}\n"
    b = "int f(int x)\n{\n  return x+1;\n}  // changed comment\n"
    c = "int f(int x) { return x + 2; }\n"
    assert bench._code_only(a) == bench._code_only(b)
    assert bench._code_only(a) != bench._code_only(c)


def _tree(tmp_path):
    src = os.path.join(ROOT, "paper_1808_08921_gb300", "csrc")
    dst = tmp_path / "paper_1808_08921_gb300" / "csrc"
    shutil.copytree(src, dst)
    return dst


def test_kernel_hash_follows_code_not_comments(tmp_path, monkeypatch):
    dst = _tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench._kernel_hash()
    f = dst / "lattice.cu"
    f.write_text(f.read_text() + "\n// a comment added at the end\n")
    assert bench._kernel_hash() == h0
    f.write_text(f.read_text() + "\nstatic int unused_probe_value = 1;\n")
    assert bench._kernel_hash() != h0
    h1 = bench._kernel_hash()
    g = dst / "api.cu"  # host-side launch code: not a profiled kernel
    g.write_text(g.read_text() + "\nstatic int unused_host_value = 1;\n")
    assert bench._kernel_hash() == h1


def test_profiled_traffic_only_for_the_profiled_code(tmp_path, monkeypatch):
    _tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    prof = tmp_path / "profile.md"
    h = bench._kernel_hash()
    prof.write_text(f"kernel_source_hash: {h}\ndram_bytes_per_launch[links]: 123000000\n")
    monkeypatch.setattr(bench, "PROFILE", str(prof))
    assert bench._profiled_traffic("links") == 123e6
    assert bench._profiled_traffic("collide_odd") is None
    prof.write_text("kernel_source_hash: 0000000000000000\ndram_bytes_per_launch[links]: 123000000\n")
    assert bench._profiled_traffic("links") is None


class _FakeStream:
    n = 0

    def __init__(self, device=None):
        _FakeStream.n += 1
        self.cuda_stream = 0x7f0000 + _FakeStream.n


class _FakeEvent:
    def __init__(self, enable_timing=False):
        self.stream = None

    def record(self, stream=None):
        self.stream = stream
        _FakeTorch.recorded.append(stream)

    def elapsed_time(self, other):
        return 6.6  # 20 steps at 0.33 ms


class _FakeCuda:
    Stream = _FakeStream
    Event = _FakeEvent

    @staticmethod
    def set_device(d):
        pass

    @staticmethod
    def synchronize():
        pass

    @staticmethod
    def current_stream():
        s = _FakeStream()
        s.cuda_stream = 0  # torch's legacy default stream
        return s

    class stream:
        def __init__(self, s):
            pass

        def __enter__(self):
            return self

        def __exit__(self, *a):
            return False


class _FakeTorch:
    cuda = _FakeCuda
    recorded = []


class _FakeSim:
    made = []

    def __init__(self, kw):
        self.kw = kw
        _FakeSim.made.append(self)

    @classmethod
    def from_workload(cls, w, **kw):
        return cls(kw)

    def step(self, n):
        pass

    def counters(self):
        return {"fluid": 4149534, "stored": 4464000, "nodes": 16777216, "links": 23875848,
                "relayouts": 0, "conversions": 0, "launches": 0}

    def set_timing(self, on):
        pass

    def timing(self):
        return {"collide_odd": (10 * 0.170, 10), "links": (10 * 0.150, 10), "map_update": (0.8, 20),
                "inlet_outlet": (0.2, 20), "dem": (0.7, 20), "collide_even": (10 * 0.200, 10)}

    def status(self):
        return 0

    def close(self):
        pass


class _FakeLbmdem:
    F32, BF16_DEV, F16_DEV = 0, 1, 2
    Sim = _FakeSim


def test_bench_runs_the_library_on_the_stream_it_times(monkeypatch, capsys):
    """The headline events must sit on the stream the library launches on:
    bench.py hands the library a dedicated non-default stream (a 0 handle
    would make the library create a private stream the events never wait
    for) and records every timing event on that same stream."""
    import argparse
    import json
    import paper_1808_08921_gb300 as pkg
    monkeypatch.setitem(sys.modules, "torch", _FakeTorch)
    monkeypatch.setitem(sys.modules, "paper_1808_08921_gb300.lbmdem", _FakeLbmdem)
    monkeypatch.setattr(pkg, "lbmdem", _FakeLbmdem, raising=False)
    _FakeSim.made.clear()
    _FakeTorch.recorded.clear()
    args = argparse.Namespace(steps=20, warmup=5, storage="f32", no_e2e=True, no_tune=True, no_cpu=True,
                              no_storage=False, no_adjoint=True, adj_steps=100, cpu_seconds=1.0)
    bench.run_ours(args)
    handles = {s.kw["cuda_stream"] for s in _FakeSim.made}
    assert len(handles) == 1 and 0 not in handles and None not in handles
    (h,) = handles
    assert _FakeTorch.recorded and all(s is not None and s.cuda_stream == h for s in _FakeTorch.recorded)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["ms_per_step"] == 0.33 and line["storage_f16"]["speedup_vs_f32"] == 1.0
    assert line["config"] == bench.workload_config(__import__("workloads").config_scale(steps=20))


def test_validate_rejects_enqueue_timed_lines():
    """The shape of a line whose events timed only the host enqueue: a step
    shorter than its own link launch and 3x the HBM roofline."""
    bad = {"value": 137779.0, "ms_per_step": 0.0301, "step_roofline": {"frac": 3.13},
           "roofline": {"us_per_launch": 153.3}}
    assert len(bench.validate(bad)) == 2
    good = {"value": 12492.0, "ms_per_step": 0.332, "step_roofline": {"frac": 0.28},
            "roofline": {"us_per_launch": 152.2}}
    assert bench.validate(good) == []
