"""Host logic of bench.py (no GPU).  The committed ncu record of the level-blocked kernel is used
only while the kernel's sources hash to the recorded value, and only for its own accumulation
and size; the algorithmic bytes and memory roofs of the line equal the byte counts of the
level-blocked and plain MPK written out by hand; clock samples are parsed as nvidia-smi prints
them; the reference arm (the CPU oracle) prints its one line on rank 0 only."""
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


class _Headline:
    """Sizes of the 256^3 7-point Laplacian: n = 256^3, nnz = 7n - 6 * 256^2."""
    n = 16_777_216
    nnz = 117_047_296


def test_algorithmic_quantities_of_the_headline(bench):
    flops, a_bytes, v_bytes = bench.algorithmic(_Headline, 8)
    assert flops == 2 * 117_047_296 * 8                     # 2 flop per stored entry and power
    assert a_bytes == 12 * 117_047_296 + 4 * 16_777_217      # A_B = (8 + 4) nnz + 4 (n + 1)
    assert v_bytes == 8 * 16_777_216                         # V = 8 n m


def test_memory_roofs_follow_the_blocked_and_plain_byte_counts(bench):
    A_B, V, n, p = 1_471_676_420, 134_217_728, 16_777_216, 8
    r = bench.memory_roofs(A_B, n, p, False, 6774.0, 18830.0)
    assert r["hbm_bytes"] == 2_679_635_972                   # A_B + (p + 1) V
    assert r["l2_bytes"] == r["plain_bytes"] == 13_920_895_008  # p (A_B + 2 V)
    t_hbm, t_l2 = 2_679_635_972 / 6774e9, 13_920_895_008 / 18830e9
    assert r["l2_blocked_roof_ms"] == pytest.approx(max(t_hbm, t_l2) * 1e3, rel=1e-12)
    assert r["plain_hbm_roof_ms"] == pytest.approx(13_920_895_008 / 6774e9 * 1e3, rel=1e-12)
    # binary32 sums over bfloat16 values: A_B = 6 nnz + 4 (n + 1); a power also writes its
    # 4-byte binary32 copy and the next one reads that copy instead of the binary64 power
    A_B16 = 6 * 117_047_296 + 4 * (n + 1)
    r = bench.memory_roofs(A_B16, n, p, True, 6774.0, 18830.0)
    assert r["hbm_bytes"] == A_B16 + 8 * n + p * 12 * n == 2_514_223_108
    assert r["l2_bytes"] == p * (A_B16 + 4 * n + 12 * n) == 8_302_624_800
    # more bandwidth never raises a roof
    assert bench.memory_roofs(A_B, n, p, False, 2 * 6774.0, 18830.0)["l2_blocked_roof_ms"] <= \
        bench.memory_roofs(A_B, n, p, False, 6774.0, 18830.0)["l2_blocked_roof_ms"]


def test_clock_summary_parses_samples_and_reasons(bench):
    clk = bench.ClockSampler(0)
    clk.lines = [
        "2070, 2070, 812.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "2055, 2070, 1390.1, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "2040, 2070, 1399.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "[N/A], 2070, [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]",   # unreadable sample: skipped
        "garbage",
    ]
    s = clk.summary()
    assert s["samples"] == 3 and s["sm_mhz"] == 2055 and s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["sw_power_cap"]
    clk.lines = ["1400, 2070, 900, 0x40, Not Active, Active, Not Active, Not Active"]
    assert clk.summary()["reasons"] == ["hw_thermal_slowdown"]
    clk.lines = []  # no nvidia-smi: no clock, the fallback maximum
    s = clk.summary()
    assert s["sm_mhz"] is None and s["samples"] == 0 and s["sm_max_mhz"] == bench.SM_MAX_MHZ_FALLBACK


def _reference_run(env_extra):
    import subprocess
    env = dict(os.environ, **env_extra)
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--side", "16", "--steps", "3",
           "--warmup", "3"]
    return subprocess.run(cmd, capture_output=True, text=True, env=env, cwd=ROOT, timeout=600)


def test_reference_arm_prints_one_line_on_rank_0_only():
    # the reference arm times the CPU oracle: rank 0 prints one JSON line with the contract's
    # keys; another rank of a multi-process launch exits 0 without work or output
    r = _reference_run({"RANK": "0", "WORLD_SIZE": "1", "LOCAL_RANK": "0"})
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["unit"] == "Gflop/s" and d["higher_is_better"] is True
    assert d["steps"] == 3 and d["value"] > 0 and d["config"]["n"] == 16 ** 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": "Gflop/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    r = _reference_run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0 and r.stdout.strip() == "", r.stderr
