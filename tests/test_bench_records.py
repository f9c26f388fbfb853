"""bench.py takes a kernel's DRAM traffic from its committed ncu record only
while the record names the SHA-256 of the current CUDA source and the same
workload; otherwise `traffic` is null with the reason.  Runs without a GPU."""
import hashlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def fake_tree(tmp_path, source=b"__global__ void k() {}\n", sha=None, m=20, n=10):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "paper_2204_00602_gb300" / "csrc").mkdir(parents=True)
    (tmp_path / "paper_2204_00602_gb300" / "csrc" / "glynn_tc.cu").write_bytes(source)
    sha = sha or hashlib.sha256(source).hexdigest()
    (tmp_path / "profiles" / "tc_product_kernel_traffic.txt").write_text(
        f"# a comment: with a colon\nsource_sha256: {sha}\nm: {m}\nn: {n}\n"
        "read_bytes: 1000\nwrite_bytes: 24\n")


def test_record_of_the_current_source_is_used(tmp_path, monkeypatch):
    fake_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    traffic, note = bench.recorded_traffic("factor_tc", 20, 10)
    assert traffic == 1024.0 and "current source" in note


def test_record_of_an_older_source_is_not_used(tmp_path, monkeypatch):
    fake_tree(tmp_path, sha="0" * 64)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    traffic, note = bench.recorded_traffic("factor_tc", 20, 10)
    assert traffic is None and "changed" in note


def test_record_of_another_workload_is_not_used(tmp_path, monkeypatch):
    fake_tree(tmp_path, m=18, n=9)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    traffic, note = bench.recorded_traffic("factor_tc", 20, 10)
    assert traffic is None and "another workload" in note


def test_missing_record_and_unrecorded_kernel(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("factor_tc", 20, 10)[0] is None
    assert bench.recorded_traffic("slos", 20, 10)[0] is None

