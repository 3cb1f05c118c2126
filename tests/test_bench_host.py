"""bench.py's host-side parts (no GPU): the reference arm's JSON line on a
tiny bounded sample, the clock-sample summary, and the guard that reports a
committed traffic figure only while the kernel sources hash the same."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "1", "--ref-crop", "12", "--ref-iters", "5"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "GLUPS"
    assert line["value"] > 0 and line["steps"] == 1 and line["warmup"] == 1 and line["higher_is_better"] is True
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and "12^3" in cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == "GLUPS"
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_clock_summary(tmp_path):
    f = tmp_path / "clocks.csv"
    f.write_text("0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                 "0, 1980, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active\n"
                 "0, 2070, 2070, 1390.2, 0x4, Not Active, Not Active, Not Active, Active\n"
                 "garbage line\n")
    c = bench.Clocks(0)
    c.proc = object()  # as if nvidia-smi had run
    c.path = str(f)
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    assert bench.Clocks(0).summary()["reasons"] == ["nvidia-smi unavailable"]


def test_traffic_figure_needs_the_same_sources(tmp_path, monkeypatch):
    good = {"kernel_source_hash": bench._kernel_source_hash(),
            "kernels": {"k_a<float, 1>": {"dram_bytes_per_cell": 12.5},
                        "k_b<float, 0>": {"dram_bytes_per_cell": 9.0},
                        "k_b<float, 1>": {"dram_bytes_per_cell": 8.0}}}
    f = tmp_path / "traffic.json"
    f.write_text(json.dumps(good))
    monkeypatch.setattr(bench, "TRAFFIC", str(f))
    assert bench._profiled_traffic("k_a<float, 1>", 10) == pytest.approx(125.0)
    assert bench._profiled_traffic("k_a", 10) == pytest.approx(125.0)  # the only instantiation
    assert bench._profiled_traffic("k_b", 10) is None  # two instantiations: ambiguous
    assert bench._profiled_traffic("k_c", 10) is None
    f.write_text(json.dumps(dict(good, kernel_source_hash="0" * 16)))
    assert bench._profiled_traffic("k_a<float, 1>", 10) is None  # taken on other sources
    monkeypatch.setattr(bench, "TRAFFIC", str(tmp_path / "missing.json"))
    assert bench._profiled_traffic("k_a<float, 1>", 10) is None



def test_batched_cpu_baseline_on_a_small_sample():
    r = bench._cpu_baseline_batched(512, sample=2)
    assert r["kind"] == "oracle" and r["unit"] == "solves/s" and r["value"] > 0 and r["cores"] >= 1
    assert "[0, 511]" in r["sample"]
    assert r["extrapolated_seconds_for_all"] == pytest.approx(512 / r["value"])


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun every rank runs bench.py; the reference arm's rank 0
    alone times the oracle and prints the line, the others exit 0 at once."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                          "--steps", "1", "--warmup", "1", "--ref-crop", "12", "--ref-iters", "5"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    assert out.stdout.strip() == ""
