"""Host logic of bench.py (CPU): the DRAM-traffic record is reported only for
the kernel sources it was captured on, the record is self-consistent, the
clock summary flags throttling, and the reference arm (the oracle) prints a
complete JSON line."""
import json
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_traffic_is_reported_only_for_the_captured_sources(monkeypatch):
    rec = json.load(open(bench.TRAFFIC_FILE))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: rec["source_hash"])
    assert bench.recorded_traffic(1000) == pytest.approx(rec["dram_bytes_per_particle"] * 1000)
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.recorded_traffic(1000) is None


def test_source_hash_covers_every_push_source(tmp_path, monkeypatch):
    h_tree = bench.kernel_source_hash()
    for p in bench.PUSH_SOURCES:
        (tmp_path / p).parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(ROOT, p), tmp_path / p)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash()
    assert h0 == h_tree
    for p in bench.PUSH_SOURCES:
        f = tmp_path / p
        orig = f.read_bytes()
        f.write_bytes(orig + b" ")
        assert bench.kernel_source_hash() != h0, p
        f.write_bytes(orig)
    assert bench.kernel_source_hash() == h0


def test_traffic_record_is_consistent():
    rec = json.load(open(bench.TRAFFIC_FILE))
    total = rec["dram_bytes_read"] + rec["dram_bytes_write"]
    assert rec["dram_bytes_per_particle"] == pytest.approx(total / rec["particles"])
    # no more than the algorithmic 24 B per particle-turn plus a few percent
    assert 0.5 * 24 < rec["dram_bytes_per_particle"] < 1.05 * 24
    assert "--clock-control none" in rec["command"]
    assert "k_push_stream" in rec["kernel"]


def _summary(tmp_path, lines):
    c = bench.ClockSampler(0)
    c.path = str(tmp_path / "clocks.csv")
    with open(c.path, "w") as f:
        f.write("\n".join(lines) + "\n")
    return c.summary()


def test_clock_summary_flags_throttle_reasons(tmp_path):
    ok = "0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active"
    cap = "0, 1980, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active"
    hot = "0, 1500, 2070, 1400.0, 0x40, Not Active, Active, Not Active, Not Active"
    s = _summary(tmp_path, [ok, ok, ok])
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 3, "source": "nvidia-smi"}
    s = _summary(tmp_path, [ok, cap, hot])
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert s["sm_mhz"] == 1980.0 and s["samples"] == 3
    s = _summary(tmp_path, [])
    assert s["samples"] == 0 and s["reasons"] == ["no nvidia-smi samples"]


class _FakeNvml:
    """Stands in for the NVML reader: a fixed sequence of (SM MHz, W, reasons)."""

    def __init__(self, rows):
        self.rows = list(rows)
        self.max_mhz = 2070.0

    def sample(self):
        return self.rows.pop(0) if self.rows else None


def test_clock_summary_from_nvml_samples(monkeypatch):
    rows = [(2070.0, 900.0, 0x0), (2055.0, 1390.0, 0x4), (1500.0, 1400.0, 0x40 | 0x4)]
    monkeypatch.setattr(bench, "_Nvml", lambda local: _FakeNvml(rows))
    with bench.ClockSampler(0) as c:
        import time
        time.sleep(0.05)
    s = c.summary()
    assert s["source"] == "nvml" and s["samples"] == 3
    assert s["sm_mhz"] == 2055.0 and s["sm_min_mhz"] == 1500.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"] and s["power_w_max"] == 1400.0


def test_reference_arm_prints_a_complete_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "mp-turns/s"
    assert d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_lane_defaults_and_flag(monkeypatch):
    """The scan and serving workloads take their measured lane counts unless
    --lanes names one (1..8, the library's range)."""
    assert set(bench.LANES) == {"l5scan", "rwscan", "hcscan", "serving"}
    assert all(1 <= v <= 8 for v in bench.LANES.values())
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", "l5scan"])
    assert bench.parse().lanes == 0   # 0: the workload's default
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", "rwscan", "--lanes", "2"])
    assert bench.parse().lanes == 2
