"""Host logic of bench.py, on CPU: the clock record taken during the timed
steps (median SM clock, maximum, throttle reasons active in any sample), the
reference arm's JSON line (the oracle timed on the host cores, the whole
step on the whole batch), the label checksum both arms print, and the order
in which the pipelined timed steps run."""
import json
import os
import subprocess
import sys
import threading
import time

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


def _record_pipeline(steps, fail_update_at=None):
    log, lock = [], threading.Lock()

    def call(kind, s):
        with lock:
            log.append((kind, s, "start", time.perf_counter()))
        time.sleep(0.02)
        if kind == "update" and s == fail_update_at:
            raise RuntimeError(f"update {s} failed")
        with lock:
            log.append((kind, s, "end", time.perf_counter()))

    err = None
    try:
        bench.run_pipelined(lambda s: call("update", s), lambda s: call("query", s), steps)
    except RuntimeError as e:
        err = e
    return log, err


def _t(log, kind, s, edge):
    return next(t for k, i, e, t in log if (k, i, e) == (kind, s, edge))


def test_pipelined_steps_order_and_overlap():
    steps = 5
    log, err = _record_pipeline(steps)
    assert err is None
    assert sorted((k, i) for k, i, e, _ in log if e == "end") == sorted(
        [("update", s) for s in range(steps)] + [("query", s) for s in range(steps)])
    for s in range(steps):
        # a step's query pass reads its own finished model
        assert _t(log, "query", s, "start") >= _t(log, "update", s, "end")
    for s in range(1, steps):
        # update s runs beside query s - 1 ...
        assert _t(log, "update", s, "start") < _t(log, "query", s - 1, "end")
        assert _t(log, "query", s - 1, "start") < _t(log, "update", s, "end")
    for s in range(2, steps):
        # ... and never overwrites the model query s - 2 was reading
        assert _t(log, "update", s, "start") >= _t(log, "query", s - 2, "end")


@pytest.mark.parametrize("steps,calls", [(0, []), (1, [("update", 0), ("query", 0)])])
def test_pipelined_steps_short_runs(steps, calls):
    log, err = _record_pipeline(steps)
    assert err is None and [(k, i) for k, i, e, _ in log if e == "start"] == calls


def test_pipelined_steps_reraise_after_the_pair():
    log, err = _record_pipeline(5, fail_update_at=2)
    assert isinstance(err, RuntimeError) and "update 2" in str(err)
    # the failing update's partner, query 1, ran to its end; nothing later started
    assert ("query", 1, "end") in [(k, i, e) for k, i, e, _ in log]
    assert not [1 for k, i, e, _ in log if e == "start" and i >= 3]
    assert ("query", 2, "start") not in [(k, i, e) for k, i, e, _ in log]
