"""The benchmark's command line and JSON line, checked without a GPU.

The reference arm times the CPU oracle, so it runs here: one JSON line with
the metric, the value, the reference marker, an end-to-end record with no
host-device bytes and a CPU-baseline record; `--capacity` reaches the
workload's configuration.  Host helpers of the engine arm are checked too.
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _reference_line(*extra):
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
           "--workload", "replay_1024x10k", "--steps", "1", "--warmup", "3", *extra]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    return json.loads(lines[0])


def test_reference_arm_json_line():
    d = _reference_line()
    assert d["impl"] == "reference"
    assert d["unit"] == "msgs/s" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["e2e"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert "sample" in cb
    # the same sample as the engine arm's cpu_baseline (every book by default)
    assert cb["sample"].startswith("first 1024 of 1024 books")
    assert cb["single_thread"]["value"] > 0 and "1 thread" in cb["single_thread"]["sample"]
    assert d["config"]["workload"] == "replay_1024x10k" and d["config"]["capacity"] == 100


def test_capacity_override_reaches_the_workload():
    d = _reference_line("--capacity", "300")
    assert d["config"]["capacity"] == 300


@pytest.mark.parametrize("cap,slots", [(1, 32), (32, 32), (33, 64), (100, 128), (128, 128),
                                       (129, 256), (250, 256), (257, 512), (500, 512)])
def test_book_bytes_follow_the_slot_count(cap, slots):
    sys.path.insert(0, ROOT)
    import bench
    # a book is two sides of 32*K slots, 24 bytes a slot (px, qty, oid, tid, time)
    assert bench.eng_book_bytes(cap) == 2 * slots * 24


def test_issue_roofline_arithmetic():
    sys.path.insert(0, ROOT)
    import bench
    # 118 warp-instructions per message at 3.89e9 messages/s on 148 SMs at
    # 2,032 MHz: 4.59e11 of 1.203e12 warp-instructions/s
    r = bench.issue_roofline(118.0, 3.89e9, 2032.0, "test", sms=148)
    assert r["bound"] == "issue"
    assert abs(r["frac"] - 118.0 * 3.89e9 / (148 * 4 * 2032e6)) < 1e-4
    assert abs(r["peak"] - 148 * 4 * 2.032) < 0.01
    assert bench.issue_roofline(None, 1.0, 2032.0, "none", sms=148)["frac"] is None
