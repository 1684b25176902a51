"""Host logic of bench.py (no GPU): the DRAM traffic of the roofline is
reported only while the kernel's source matches the hash the ncu record was
taken with, and only for the recorded workload; the BF16 peak comes from the
measured-peaks file when present."""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _tree(tmp_path, src_text, record_sha, workload="w_bf16", nbytes=1234):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "k.cu").write_text(src_text)
    (tmp_path / "profiles" / "roofline_traffic.txt").write_text(
        "# kernel sha bytes workload\n" f"my_kernel {record_sha} {nbytes} {workload}\n")


def test_traffic_reported_only_for_the_recorded_source_and_workload(tmp_path, monkeypatch):
    src = "__global__ void k() {}\n"
    sha = hashlib.sha256(src.encode()).hexdigest()[:12]
    _tree(tmp_path, src, sha)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._recorded_traffic("my_kernel", "k.cu", "w_bf16") == 1234
    assert bench._recorded_traffic("my_kernel", "k.cu", "other_bf16") is None
    assert bench._recorded_traffic("other_kernel", "k.cu", "w_bf16") is None
    (tmp_path / "k.cu").write_text(src + "// changed\n")
    assert bench._recorded_traffic("my_kernel", "k.cu", "w_bf16") is None


def test_missing_record_gives_no_traffic(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._recorded_traffic("my_kernel", "k.cu", "w_bf16") is None


def test_bf16_peak_from_the_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peak, src = bench._bf16_peak()
    assert src.startswith("fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"bf16_tflops_sustained": 1234.5}))
    peak, src = bench._bf16_peak()
    assert peak == 1234.5 and src.startswith("measured")
