"""The oracle's pins must catch plausible mistakes.  Each case copies the
oracle source to a temporary directory, plants ONE mistake (a dropped term, a
wrong sign, a wrong index or comparison), compiles it there, and checks that
the hand-worked examples reject it: the book examples for the matching rules,
the hand-worked environment episodes (rewards as literal float32 bits) for the
reward of eqs. rewardfunc / vwap.  Nothing is planted in the real oracle."""
import ctypes
import itertools
import os
import subprocess

import numpy as np
import pytest

import oracle
from golden_format import cases, side_rows, trade_rows
from test_env_oracle import ENV_FIXTURES, load_env_fixture, reward_bits

HERE = os.path.dirname(os.path.abspath(__file__))

SRC = os.path.join(os.path.dirname(oracle.__file__), "lob_oracle.cpp")

MUTANTS = {
    "fill_sign": ("std::max(0, Q_s - Q_a)", "std::max(0, Q_a - Q_s)"),
    "trade_qty_term": ("t.qty = Q_s - Q_s_new;", "t.qty = Q_s;"),
    "trade_price_from_aggressor": ("t.price = s.price;", "t.price = P_a;"),
    "cross_strict": ("(P_a <= s.price) : (P_a >= s.price)", "(P_a < s.price) : (P_a > s.price)"),
    "bid_best_is_min": ("return is_bid ? levels.rbegin()->second : levels.begin()->second;",
                        "return levels.begin()->second;"),
    "cancel_keeps_zero": ("if (q_new <= 0) {  // Q <= 0", "if (q_new < 0) {  // Q <= 0"),
    "lifo_in_level": ("Order& best() { return best_level().front(); }",
                      "Order& best() { return best_level().back(); }"),
    "evict_on_equal": ("own.strictly_better(m.price, own.worst().price)",
                       "!own.strictly_better(own.worst().price, m.price)"),
    "market_rests": ("bk.counters[C_MARKET_DISCARDED_QTY] += rest;",
                     "bk.counters[C_MARKET_DISCARDED_QTY] += rest; if (rest > 0) add(E, bk, m, rest);"),
}


# mistakes in the environment's reward (Sec. 5.2.4): each changes at least one
# hand-worked reward of the two golden episodes
REWARD_MUTANTS = {
    "advantage_sign": ("(double)sums.apq - (double)sums.aq * vwap;",
                       "(double)sums.aq * vwap - (double)sums.apq;"),
    "advantage_uses_all_trades_qty": ("(double)sums.apq - (double)sums.aq * vwap;",
                                      "(double)sums.apq - (double)sums.sq * vwap;"),
    "vwap_over_agent_trades": ("(double)sums.spq / (double)sums.sq;",
                               "(double)sums.apq / (double)sums.aq;"),
    "drift_sign": ("(vwap - es.p_init)", "(es.p_init - vwap)"),
    "drift_drops_quantity": ("cfg.lambda * ((double)sums.aq * (vwap - es.p_init))",
                             "cfg.lambda * (vwap - es.p_init)"),
}


# mistakes in snapshot initialisation and the snapshot cancel rule (Sec. 5.1.1)
SNAPSHOT_MUTANTS = {
    "snapshot_cancel_strict": ("if (q.oid <= SNAPSHOT_OID_MAX) {", "if (q.oid < SNAPSHOT_OID_MAX) {"),
    "snapshot_cancel_takes_latest": ("""                if (q.oid <= SNAPSHOT_OID_MAX) {
                    o = &q;
                    break;
                }""", """                if (q.oid <= SNAPSHOT_OID_MAX) {
                    o = &q;
                }"""),
    "snapshot_cancel_any_order": ("if (q.oid <= SNAPSHOT_OID_MAX) {", "if (true) {"),
    "init_first_oid": ("int32_t next_oid = -9000;", "int32_t next_oid = -9001;"),
    "init_oids_count_up": ("next_oid--, 0, time_ns", "next_oid++, 0, time_ns"),
    "init_ignores_zero_volume": ("px[listed] > 0 && qty[listed] > 0", "px[listed] > 0"),
}


def _build_mutant(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, name
    path = tmp_path / ("%s.cpp" % name)
    path.write_text(src.replace(old, new))
    so = tmp_path / ("lib%s.so" % name)
    subprocess.run(["g++", "-O1", "-std=c++17", "-fPIC", "-shared", "-pthread", "-o", str(so),
                    str(path)], check=True, capture_output=True)
    return str(so)


def _golden_ok(lib):
    vp, i32 = ctypes.c_void_p, ctypes.c_int32
    lib.oracle_create.restype = vp
    lib.oracle_create.argtypes = [i32] * 5
    lib.oracle_process.restype = ctypes.c_int64
    lib.oracle_process.argtypes = [vp, vp, vp, vp, i32, i32]
    lib.oracle_get_book.argtypes = [vp] * 7
    lib.oracle_get_trades.argtypes = [vp] * 3
    lib.oracle_destroy.argtypes = [vp]
    for c in cases():
        h = lib.oracle_create(1, c.capacity, c.trade_capacity, c.rule, 0)
        m = c.message_array()
        off = np.array([0, len(m)], np.int64)
        lib.oracle_process(h, vp(m.ctypes.data), vp(off.ctypes.data), None, 1, 1)
        shp = (1, 2, c.capacity)
        px, qty, oid, tid = (np.empty(shp, np.int32) for _ in range(4))
        tm = np.empty(shp, np.int64)
        cnt = np.empty((1, 2), np.int32)
        lib.oracle_get_book(h, *[vp(a.ctypes.data) for a in (px, qty, oid, tid, tm, cnt)])
        tr = np.empty((1, c.trade_capacity), oracle.TRADE_DTYPE)
        tc = np.empty(1, np.int64)
        lib.oracle_get_trades(h, vp(tr.ctypes.data), vp(tc.ctypes.data))
        lib.oracle_destroy(h)
        bk = dict(price=px, qty=qty, oid=oid, tid=tid, time_ns=tm, count=cnt)
        if (side_rows(bk, 0, 0) != c.bids or side_rows(bk, 0, 1) != c.asks
                or trade_rows(tr, tc, 0, c.trade_capacity) != c.trades
                or int(tc[0]) != c.trades_total):
            return False
    return True


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_golden_examples_reject_mutant(tmp_path, name):
    old, new = MUTANTS[name]
    lib = ctypes.CDLL(_build_mutant(tmp_path, name, old, new))
    assert not _golden_ok(lib), "planted mistake %r went unnoticed" % name


def test_unmutated_copy_passes(tmp_path):
    lib = ctypes.CDLL(_build_mutant(tmp_path, "identity", "int oracle_abi_version(void) { return 1; }",
                                    "int oracle_abi_version(void) { return 1; }"))
    assert _golden_ok(lib)


def _env_golden_ok(lib):
    """Run both hand-worked episodes (lambda 0 and 1/2) through a compiled
    oracle and compare every reward's bits with the literal ones."""
    vp, i32 = ctypes.c_void_p, ctypes.c_int32
    lib.oracle_env_create.restype = vp
    lib.oracle_env_create.argtypes = [i32] * 10 + [ctypes.c_double]
    lib.oracle_env_step.argtypes = [vp, vp, vp, vp, vp, i32] + [vp] * 6 + [i32, vp]
    lib.oracle_env_destroy.argtypes = [vp]
    for fx in ENV_FIXTURES:
        cfg, steps, _, _ = load_env_fixture(os.path.join(HERE, "golden", fx))
        for lam in (0.0, 0.5):
            h = lib.oracle_env_create(1, cfg["capacity"], 64, cfg["n_steps"], cfg["parent"],
                                      cfg["agent_tid"], cfg["depth"], cfg["p_init_fallback"], 2, 1,
                                      lam)
            ok = True
            for st in steps:
                m = oracle.messages(st["msgs"])
                off = np.array([0, len(m)], np.int64)
                draw = np.array([st["draw"]], np.uint32)
                reward = np.empty(1, np.float32)
                lv = [np.empty((1, cfg["depth"]), np.int32) for _ in range(4)]
                fills = np.empty((1, 2), np.int64)
                lib.oracle_env_step(h, vp(m.ctypes.data), vp(off.ctypes.data),
                                    vp(draw.ctypes.data), None, st["step"],
                                    vp(reward.ctypes.data), *[vp(x.ctypes.data) for x in lv],
                                    vp(fills.ctypes.data), 1, None)
                ok = ok and reward_bits(reward[0]) == st["reward"][lam]
            lib.oracle_env_destroy(h)
            if not ok:
                return False
    return True


@pytest.mark.parametrize("name", sorted(REWARD_MUTANTS))
def test_env_golden_episodes_reject_reward_mutant(tmp_path, name):
    old, new = REWARD_MUTANTS[name]
    lib = ctypes.CDLL(_build_mutant(tmp_path, name, old, new))
    assert not _env_golden_ok(lib), "planted reward mistake %r went unnoticed" % name


def test_unmutated_copy_passes_env_episodes(tmp_path):
    lib = ctypes.CDLL(_build_mutant(tmp_path, "identity_env",
                                    "int oracle_abi_version(void) { return 1; }",
                                    "int oracle_abi_version(void) { return 1; }"))
    assert _env_golden_ok(lib)


def _snapshot_golden_ok(lib):
    """The hand-worked snapshot cases of tests/test_snapshot_init.py, run
    through a compiled oracle: initialisation of three books, and the
    price-matched cancels (one snapshot order per level, and two at one
    price)."""
    import test_snapshot_init as ts
    vp, i32 = ctypes.c_void_p, ctypes.c_int32
    lib.oracle_create.restype = vp
    lib.oracle_create.argtypes = [i32] * 5
    lib.oracle_destroy.argtypes = [vp]
    lib.oracle_init_from_levels.restype = i32
    lib.oracle_init_from_levels.argtypes = [vp] * 5 + [i32, ctypes.c_int64]
    lib.oracle_process.restype = ctypes.c_int64
    lib.oracle_process.argtypes = [vp, vp, vp, vp, i32, i32]
    lib.oracle_get_book.argtypes = [vp] * 7

    def book(h, n, cap):
        shp = (n, 2, cap)
        out = {k: np.empty(shp, np.int32) for k in ("price", "qty", "oid", "tid")}
        out["time_ns"] = np.empty(shp, np.int64)
        out["count"] = np.empty((n, 2), np.int32)
        lib.oracle_get_book(h, *[vp(out[k].ctypes.data) for k in
                                 ("price", "qty", "oid", "tid", "time_ns", "count")])
        return out

    def init(h, levels, t=0):
        a = [np.ascontiguousarray(x, np.int32) for x in levels]
        return lib.oracle_init_from_levels(h, *[vp(x.ctypes.data) for x in a], a[0].shape[1], t)

    def run(h, rows):
        m = ts._msg(rows)
        off = np.array([0, len(m)], np.int64)
        lib.oracle_process(h, vp(m.ctypes.data), vp(off.ctypes.data), None, 1, 1)

    ok = True
    h = lib.oracle_create(3, 4, 8, 0, 0)
    ok &= init(h, ts._levels_case(), 77) == 1
    bk = book(h, 3, 4)
    ok &= all(bk[k].tolist() == v for k, v in ts.HAND_INIT.items())
    lib.oracle_destroy(h)
    # one snapshot order per level (the cancel-rule example)
    h = lib.oracle_create(1, 8, 16, 0, 2)
    init(h, (np.array([[100, 99]]), np.array([[5, 7]]), np.array([[101, 103]]),
             np.array([[4, 6]])))
    run(h, [(2, ts.BID, 99, 3, 555), (3, ts.ASK, 103, 6, 777), (2, ts.BID, 98, 1, 888),
            (2, ts.BID, 101, 1, 889), (1, ts.BID, 99, 2, 10), (2, ts.BID, 99, 4, 556),
            (2, ts.BID, 99, 1, 557), (2, ts.BID, 99, 1, 10), (2, ts.BID, 100, 1, 558)])
    bk = book(h, 1, 8)
    ok &= bk["oid"][0, 0, :2].tolist() == [-9000, 10] and bk["qty"][0, 0, :2].tolist() == [4, 1]
    ok &= bk["count"][0].tolist() == [2, 1]
    lib.oracle_destroy(h)
    # two snapshot orders at one price
    h = lib.oracle_create(1, 8, 16, 0, 2)
    init(h, (np.array([[100, 100, 99]]), np.array([[5, 3, 7]]), np.array([[101, 102, 103]]),
             np.array([[4, 4, 4]])))
    run(h, [(2, ts.BID, 100, 2, 555), (3, ts.BID, 100, 3, 556), (2, ts.BID, 100, 1, 557)])
    bk = book(h, 1, 8)
    ok &= bk["oid"][0, 0, :2].tolist() == [-9001, -9002] and bk["qty"][0, 0, :2].tolist() == [2, 7]
    lib.oracle_destroy(h)
    return bool(ok)


@pytest.mark.parametrize("name", sorted(SNAPSHOT_MUTANTS))
def test_snapshot_examples_reject_mutant(tmp_path, name):
    old, new = SNAPSHOT_MUTANTS[name]
    lib = ctypes.CDLL(_build_mutant(tmp_path, name, old, new))
    assert not _snapshot_golden_ok(lib), "planted snapshot mistake %r went unnoticed" % name


def test_unmutated_copy_passes_snapshot_examples(tmp_path):
    lib = ctypes.CDLL(_build_mutant(tmp_path, "identity_snap",
                                    "int oracle_abi_version(void) { return 1; }",
                                    "int oracle_abi_version(void) { return 1; }"))
    assert _snapshot_golden_ok(lib)
