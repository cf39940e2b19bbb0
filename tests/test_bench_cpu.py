"""bench.py on the CPU: the reference arm (the oracle timed on the host
cores) prints one JSON line with the keys the measurement contract names,
and the clock summary reads nvidia-smi's sampled lines (median SM clock
under load, the throttle reasons seen) inside the timed window only."""
import importlib.util
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_reference_arm_prints_one_contract_line(orc):
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "1", "--cpu-freqs", "2"], cwd=ROOT, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["unit"] == "GB/s" and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert 0.2 < d["ratio"] < 0.6


def test_clock_summary_keeps_the_window_and_the_reasons():
    b = load_bench()
    c = b.ClockSampler(0)
    row = "{sm}, 2070, 900.5, 0x0, {hw}, Not Active, Not Active, {pc}"
    c.lines = [(1.0, row.format(sm=1200, hw="Not Active", pc="Not Active")),   # before
               (2.0, row.format(sm=2070, hw="Not Active", pc="Active")),
               (2.1, row.format(sm=2040, hw="Not Active", pc="Not Active")),
               (2.2, row.format(sm=2070, hw="Not Active", pc="Not Active")),
               (3.5, row.format(sm=900, hw="Active", pc="Not Active")),        # after
               (2.3, "[N/A], garbled")]
    s = b.ClockSampler.summary(c, 1.5, 3.0)
    assert s["samples"] == 3 and s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    empty = b.ClockSampler.summary(c, 10.0, 11.0)
    assert empty["samples"] == 0 and empty["sm_mhz"] is None


def test_recorded_profile_is_tied_to_the_kernel_sources(tmp_path, monkeypatch):
    b = load_bench()
    assert len(b.kernel_source_hash()) == 16      # the real sources hash
    rec = {"source_hash": "5eed5eed5eed5eed", "units_per_launch": 100,
           "dram_bytes_per_launch": 1000.0, "inst_per_launch": 50.0}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    monkeypatch.setattr(b, "kernel_source_hash", lambda: "5eed5eed5eed5eed")
    assert b.recorded_profile(300) == pytest.approx(3000.0)
    assert b.recorded_profile(300, key="inst_per_launch") == pytest.approx(150.0)
    rec["source_hash"] = "0" * 16
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    assert b.recorded_profile(300) is None
