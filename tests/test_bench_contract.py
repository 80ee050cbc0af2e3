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

import numpy as np
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


def _env_episode(n, steps, w, params, ids, draws=None, actions=None):
    """Host arrays of one episode of the oracle's environments (the shape of
    the device outputs the bench compares) and its final books and state."""
    import lobgen
    import oracle
    per = w["msgs_per_step"]
    hm, _ = lobgen.generate(params, [steps * per] * n, stream_ids=ids)
    rows = hm.reshape(n, steps, per)
    oenv = oracle.EnvOracle(n, w["capacity"], 4096, n_steps=steps)
    got = dict(reward=[], bid_px=[], bid_qty=[], ask_px=[], ask_qty=[], fills=[])
    tr = None
    for t in range(steps):
        stp = np.ascontiguousarray(rows[:, t, :]).reshape(-1)
        offs = np.arange(0, n * per + 1, per)
        if actions is None:
            r_, lv, f_ = oenv.step(stp, offs, draws[t], t)
        else:
            r_, lv, f_, tr = oenv.step(stp, offs, None, t, l1=True, actions=actions[t])
        got["reward"].append(r_)
        got["fills"].append(f_)
        for k, x in zip(("bid_px", "bid_qty", "ask_px", "ask_qty"), lv):
            got[k].append(x)
    got = {k: np.stack(v) for k, v in got.items()}
    st, p0 = oenv.state()
    final = dict(state=st, p_init=p0, books=oenv.books.book())
    obs = oenv.observe(tr, per, rows[:, 0, 0]["time_ns"].astype(np.int64)) if tr is not None \
        else None
    return got, final, obs


def test_env_oracle_check_passes_the_oracles_episode_and_fails_a_changed_one():
    """The bench's all-environments RL parity check, chunked (3 chunks, the
    last ragged): equal outputs pass; one reward bit, one fill or one final
    book entry changed fails; the policy form's observation is checked too."""
    sys.path.insert(0, ROOT)
    import bench
    import lobgen
    w = dict(lobgen.WORKLOADS["rl_exec_8192x400"])
    n, steps = 9, 12
    params = lobgen.make_params(w["seed"], w["mid_walk"])
    ids = np.arange(n, dtype=np.uint64)
    draws = lobgen.agent_draws(w["seed"] + 1, n, steps)
    got, final, _ = _env_episode(n, steps, w, params, ids, draws=draws)
    assert bench.env_oracle_check(w, params, ids, got, draws=draws, final=final, chunk=4)
    bad = {k: v.copy() for k, v in got.items()}
    bad["reward"][steps - 1, n - 1] = np.nextafter(bad["reward"][steps - 1, n - 1], np.float32(1e9))
    assert not bench.env_oracle_check(w, params, ids, bad, draws=draws, chunk=4)
    bad = {k: v.copy() for k, v in got.items()}
    bad["fills"][3, 5, 0] += 1
    assert not bench.env_oracle_check(w, params, ids, bad, draws=draws, chunk=4)
    fb = dict(final, books={k: v.copy() for k, v in final["books"].items()})
    fb["books"]["qty"][8, 0, 0] += 1
    assert not bench.env_oracle_check(w, params, ids, got, draws=draws, final=fb, chunk=4)
    rng = np.random.default_rng(3)
    act = (rng.random((steps, n, 4)) * 4.0).astype(np.float32)
    got, _, obs = _env_episode(n, steps, w, params, ids, actions=act)
    assert bench.env_oracle_check(w, params, ids, got, actions=act, obs=obs, chunk=4) == (True, True)
    ob = obs.copy()
    ob[7, 0] += 1.0
    assert bench.env_oracle_check(w, params, ids, got, actions=act, obs=ob, chunk=4) == (True, False)


class _OracleAsEngine:
    """The outputs the bench reads from an engine, served by an oracle run
    (CPU torch tensors), optionally with one value changed."""

    def __init__(self, o, depth=10, change=None):
        import torch
        self.bk = {k: torch.from_numpy(v.copy()) for k, v in o.book().items()}
        self.lv = [torch.from_numpy(x.copy()) for x in o.levels(depth)]
        self.ctr = torch.from_numpy(o.counters().copy())
        tr, cnt = o.trades()
        self.tr = torch.from_numpy(tr.view(np.int32).reshape(o.n_books, o.trade_capacity, 8).copy())
        self.cnt = torch.from_numpy(cnt.copy())
        if change == "level":
            self.lv[3][5, 0] += 1
        elif change == "trade_log":
            self.tr[1, 0, 1] += 1
        elif change == "count":
            self.cnt[6] += 1

    def book(self):
        return self.bk

    def levels(self, depth):
        return self.lv

    def stats(self):
        import torch
        return self.ctr, torch.zeros(1, dtype=torch.int32)

    def trades(self):
        return self.tr, self.cnt


@pytest.mark.parametrize("change", [None, "level", "trade_log", "count"])
def test_replay_oracle_check_every_book_in_chunks(change):
    """The bench's every-book replay check (3 chunks, the last ragged): the
    oracle's own outputs pass; a changed level, trade-log entry of a checked
    log or trade count fails."""
    sys.path.insert(0, ROOT)
    import bench
    import lobgen
    import oracle
    n, cap, tcap = 7, 100, 400
    params = lobgen.make_params(5, "pm1")
    ids = np.arange(n, dtype=np.uint64)
    counts = np.array([300, 10, 700, 0, 250, 500, 90], dtype=np.int64)
    m, off = lobgen.generate(params, counts, stream_ids=ids)
    o = oracle.Oracle(n, cap, tcap)
    o.process(m, off)
    ok, _ = bench.replay_oracle_check(_OracleAsEngine(o, change=change), params, ids, counts, cap,
                                      tcap, chunk=3, logs=2)
    assert ok == (change is None)
