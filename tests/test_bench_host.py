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


def test_profiled_traffic_only_for_the_profiled_code(tmp_path, monkeypatch):
    _tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    prof = tmp_path / "profile.md"
    h = bench._kernel_hash()
    prof.write_text(f"kernel_source_hash: {h}\ndram_bytes_per_launch[links]: 123000000\n")
    monkeypatch.setattr(bench, "PROFILE", str(prof))
    assert bench._profiled_traffic("links") == 123e6
    assert bench._profiled_traffic("collide_stream") is None
    prof.write_text("kernel_source_hash: 0000000000000000\ndram_bytes_per_launch[links]: 123000000\n")
    assert bench._profiled_traffic("links") is None
