"""Host logic of bench.py, on CPU: the clock record taken during the timed
steps (median SM clock, maximum, throttle reasons active in any sample) and
the reference arm's JSON line (the oracle timed on the host cores, the whole
step on the whole batch), and the label checksum both arms print."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _sampler(lines, t0=100.0):
    s = bench.ClockSampler()
    s.t0 = t0
    s.samples = [(t, [x.strip() for x in line.split(",")]) for t, line in lines]
    return s


def test_clock_record_median_max_and_reasons():
    na, act = "Not Active", "Active"
    s = _sampler([
        (99.0, f"900, 2070, 300, 0x0, {act}, {na}, {na}, {na}"),  # before the timed region: ignored
        (100.1, f"2070, 2070, 900, 0x0, {na}, {na}, {na}, {na}"),
        (100.2, f"2040, 2070, 1300, 0x4, {na}, {na}, {na}, {act}"),
        (100.3, f"1980, 2070, 1390, 0x4, {na}, {na}, {na}, {act}"),
    ])
    rec = s.stop()
    assert rec["samples"] == 3
    assert rec["sm_mhz"] == 2040.0 and rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"]


def test_clock_record_reports_every_slowdown_kind():
    na, act = "Not Active", "Active"
    s = _sampler([(101.0, f"1500, 2070, 1400, 0x68, {act}, {act}, {act}, {na}")])
    assert s.stop()["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_record_without_samples():
    rec = _sampler([]).stop()
    assert rec["samples"] == 0 and rec["sm_mhz"] is None and rec["reasons"] == ["unavailable"]
    # only a sample from before the timed region: the last one stands in
    rec = _sampler([(50.0, "2070, 2070, 500, 0x0, Not Active, Not Active, Not Active, Not Active")]).stop()
    assert rec["samples"] == 1 and rec["sm_mhz"] == 2070.0 and rec["reasons"] == []


def test_reference_arm_prints_one_contract_line():
    # a smaller batch than the default 4,194,304 keeps the CPU suite short
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--queries", "65536"], cwd=ROOT, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "checks/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["ms_per_step"] == pytest.approx(65536 / d["value"] * 1e3)
    assert d["config"]["n_query"] == 65536
    assert d["labels_checksum"]["positive"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "checks/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "arm7-n5000" and d["data"] == "synthetic"


def test_label_checksum_sees_every_label():
    import numpy as np
    a = np.where(np.arange(1000) % 3 == 0, 1, -1).astype(np.int8)
    b = a.copy()
    b[500], b[501] = b[501], b[500]  # same count, two labels swapped
    ca, cb = bench.label_checksum(a), bench.label_checksum(b)
    assert ca["positive"] == cb["positive"] and ca["weighted"] != cb["weighted"]
    assert bench.label_checksum(a) == ca
