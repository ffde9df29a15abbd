"""Host logic of bench.py (no GPU): the committed ncu record of the level-blocked kernel is used
only while the kernel's sources hash to the recorded value, and only for its own accumulation
and size."""
import hashlib
import importlib.util
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture()
def bench(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _record(tmp_path, bench, sha, side=256):
    rec = {"kernel_source_sha256": sha,
           "records": {"f64": {"side": side, "dram_bytes_per_launch": 123, "l2_hit_rate": 0.5},
                       "f32": {"side": side, "dram_bytes_per_launch": 456, "l2_hit_rate": 0.4}}}
    path = tmp_path / "traffic.json"
    path.write_text(json.dumps(rec))
    return str(path)


def _sources_sha(paths):
    h = hashlib.sha256()
    for f in paths:
        h.update(open(f, "rb").read())
    return h.hexdigest()


def test_record_used_while_the_sources_match(bench, tmp_path, monkeypatch):
    srcs = []
    for i, text in enumerate((b"kernel", b"header", b"planner")):
        f = tmp_path / f"src{i}"
        f.write_bytes(text)
        srcs.append(str(f))
    monkeypatch.setattr(bench, "KERNEL_SOURCES", srcs)
    monkeypatch.setattr(bench, "TRAFFIC_RECORD", _record(tmp_path, bench, _sources_sha(srcs)))
    assert bench.measured_profile(256, "f64")["dram_bytes_per_launch"] == 123
    assert bench.measured_profile(256, "f32")["l2_hit_rate"] == 0.4
    assert bench.measured_profile(128, "f64") is None  # another workload size
    assert bench.measured_profile(256, "bf16") is None  # no record for that case
    (tmp_path / "src1").write_bytes(b"header, changed")
    assert bench.measured_profile(256, "f64") is None  # the kernel changed since the capture


def test_missing_or_broken_record(bench, tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "TRAFFIC_RECORD", str(tmp_path / "absent.json"))
    assert bench.measured_profile(256, "f64") is None
    bad = tmp_path / "bad.json"
    bad.write_text("{not json")
    monkeypatch.setattr(bench, "TRAFFIC_RECORD", str(bad))
    assert bench.measured_profile(256, "f64") is None


def test_committed_record_names_its_sources(bench):
    rec = json.load(open(bench.TRAFFIC_RECORD))
    assert set(rec["records"]) == {"f64", "f32"}
    assert [os.path.normpath(os.path.join(ROOT, f)) for f in rec["hashed_files"]] == \
        [os.path.normpath(f) for f in bench.KERNEL_SOURCES]
    for case in rec["records"].values():
        assert case["dram_bytes_per_launch"] > case["measured"]["algorithmic_min_bytes"]
