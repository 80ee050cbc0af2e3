"""CPU oracle for the limit-order-book engine -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg may import this package.  The engine (``paper_2308_13289_b300``)
never imports it, and the two share no code: the only common module is the
seeded input generator ``lobgen``, which holds no order-book arithmetic.

Two independent CPU implementations live here:

* ``lob_oracle.cpp`` (class :class:`Oracle`): the plain definition of
  price-time-priority matching from Sec. 4.1-4.2 with an ordered map of
  per-price FIFO queues.  This is the oracle the GPU is compared with.
* ``lob_literal.c`` (:func:`literal_run`): the paper's own unsorted-array
  formulation (Sec. 4 eqs. 1-2, Sec. 4.1), used only to cross-check the oracle
  by brute force on tiny books.

``lob_oracle.cpp`` also holds (class :class:`EnvOracle`) the execution-environment
step of Sec. 5 (replay, then the synthetic agent's orders, top levels, agent
fills and the VWAP reward of eqs. rewardfunc / vwap).

Parity status: matching, cancel, dispatch, levels and the canonical dump are
pinned by hand-worked examples, closed forms, invariants and the brute-force
cross-check; the full-side rule, the trade-log bound, the synthetic agent, the
reward's handling of empty steps, the snapshot OIDs' order and the <= -9000
reading, the action map's rounding and sizing, and the observation's values
for a missing side are readings of silent or conflicting passages, pinned
only by hand-worked examples (parity against the paper itself unpinned there).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ORACLE_SO = os.path.join(HERE, "liblob_oracle.so")
LITERAL_SO = os.path.join(HERE, "liblob_literal.so")

MSG_DTYPE = np.dtype([("type", "<i4"), ("side", "<i4"), ("price", "<i4"), ("qty", "<i4"),
                      ("oid", "<i4"), ("tid", "<i4"), ("time_ns", "<i8")])
TRADE_DTYPE = np.dtype([("price", "<i4"), ("qty", "<i4"), ("oid_aggr", "<i4"),
                        ("oid_stand", "<i4"), ("tid_aggr", "<i4"), ("tid_stand", "<i4"),
                        ("time_ns", "<i8")])

COUNTERS = ["msgs", "limit", "cancel", "market", "noop", "invalid", "trades", "traded_qty",
            "rested", "rejected", "rejected_qty", "evicted", "evicted_qty", "cancel_hit",
            "cancelled_qty", "cancel_miss", "market_discarded_qty", "limit_qty", "market_qty",
            "trades_dropped"]


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("oracle build failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))


def build(force: bool = False) -> None:
    """Compile the CPU oracle libraries (g++/gcc, no FMA contraction)."""
    jobs = [
        (ORACLE_SO, ["lob_oracle.cpp"], ["g++", "-O2", "-std=c++17"]),
        (LITERAL_SO, ["lob_literal.c"], ["gcc", "-O2", "-std=c11"]),
    ]
    for so, srcs, cc in jobs:
        paths = [os.path.join(HERE, s) for s in srcs]
        if not all(os.path.exists(p) for p in paths):
            continue
        newest = max(os.path.getmtime(p) for p in paths)
        if force or not os.path.exists(so) or os.path.getmtime(so) < newest:
            _run(cc + ["-fPIC", "-shared", "-pthread", "-ffp-contract=off", "-o", so] + paths)


_libs = {}


def _lib(path):
    if path not in _libs:
        if not os.path.exists(path):
            build()
        _libs[path] = ctypes.CDLL(path)
    return _libs[path]


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _oracle_lib():
    lib = _lib(ORACLE_SO)
    vp, i32 = ctypes.c_void_p, ctypes.c_int32
    lib.oracle_create.restype = vp
    lib.oracle_create.argtypes = [i32, i32, i32, i32, i32]
    lib.oracle_destroy.argtypes = [vp]
    lib.oracle_process.restype = ctypes.c_int64
    lib.oracle_process.argtypes = [vp, vp, vp, vp, i32, i32]
    lib.oracle_process_l1.restype = ctypes.c_int64
    lib.oracle_process_l1.argtypes = [vp, vp, vp, vp, i32, i32, vp]
    lib.oracle_clear_trades.argtypes = [vp]
    lib.oracle_get_trades.argtypes = [vp, vp, vp]
    lib.oracle_get_book.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    lib.oracle_set_book.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    lib.oracle_init_from_levels.restype = i32
    lib.oracle_init_from_levels.argtypes = [vp, vp, vp, vp, vp, i32, ctypes.c_int64]
    lib.oracle_get_levels.argtypes = [vp, i32, vp, vp, vp, vp]
    lib.oracle_get_counters.argtypes = [vp, vp]
    lib.oracle_get_resting_qty.argtypes = [vp, vp]
    assert lib.oracle_n_counters() == len(COUNTERS)
    return lib


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


class Oracle:
    """n_books independent books; the same call sequence as the engine's C ABI."""

    def __init__(self, n_books: int, capacity: int, trade_capacity: int,
                 overflow_rule: int = 0, append_trades: bool = False, _borrow=None,
                 snapshot_cancels: bool = False):
        self.lib = _oracle_lib()
        self.n_books, self.capacity, self.trade_capacity = n_books, capacity, trade_capacity
        if _borrow is not None:  # books owned by an EnvOracle
            self.h, self._owned = _borrow, False
            return
        self._owned = True
        self.h = self.lib.oracle_create(n_books, capacity, trade_capacity, overflow_rule,
                                        (1 if append_trades else 0) |
                                        (2 if snapshot_cancels else 0))
        if not self.h:
            raise ValueError("invalid oracle configuration")

    def __del__(self):
        h = getattr(self, "h", None)
        if h and getattr(self, "_owned", False):
            self.lib.oracle_destroy(h)
            self.h = None

    def process(self, msgs: np.ndarray, offsets: np.ndarray, book_ids=None, threads=None):
        msgs = np.ascontiguousarray(msgs, dtype=MSG_DTYPE)
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        ids = None if book_ids is None else np.ascontiguousarray(book_ids, dtype=np.int32)
        n_active = len(offsets) - 1
        if ids is None and n_active != self.n_books:
            raise ValueError("without book_ids every book needs a segment")
        err = self.lib.oracle_process(self.h, _p(msgs) if len(msgs) else None, _p(offsets),
                                      _p(ids), n_active, threads or default_threads())
        if err:
            raise RuntimeError("oracle: %d duplicate live OIDs (contract violation)" % err)

    def process_l1(self, msgs: np.ndarray, offsets: np.ndarray, book_ids=None, threads=None):
        """process() and return the level-1 state after every message:
        int32 [len(msgs), 4] = bid price, bid qty, ask price, ask qty."""
        msgs = np.ascontiguousarray(msgs, dtype=MSG_DTYPE)
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        ids = None if book_ids is None else np.ascontiguousarray(book_ids, dtype=np.int32)
        n_active = len(offsets) - 1
        l1 = np.full((len(msgs), 4), -7, np.int32)
        err = self.lib.oracle_process_l1(self.h, _p(msgs) if len(msgs) else None, _p(offsets),
                                         _p(ids), n_active, threads or default_threads(),
                                         _p(l1) if len(msgs) else None)
        if err:
            raise RuntimeError("oracle: %d duplicate live OIDs (contract violation)" % err)
        return l1

    def clear_trades(self):
        self.lib.oracle_clear_trades(self.h)

    def trades(self):
        out = np.empty((self.n_books, self.trade_capacity), dtype=TRADE_DTYPE)
        cnt = np.empty(self.n_books, dtype=np.int64)
        self.lib.oracle_get_trades(self.h, _p(out), _p(cnt))
        return out, cnt

    def book(self):
        shp = (self.n_books, 2, self.capacity)
        px, qty, oid, tid = (np.empty(shp, np.int32) for _ in range(4))
        tm = np.empty(shp, np.int64)
        cnt = np.empty((self.n_books, 2), np.int32)
        self.lib.oracle_get_book(self.h, _p(px), _p(qty), _p(oid), _p(tid), _p(tm), _p(cnt))
        return dict(price=px, qty=qty, oid=oid, tid=tid, time_ns=tm, count=cnt)

    def set_book(self, bk: dict):
        dt = dict(price=np.int32, qty=np.int32, oid=np.int32, tid=np.int32, time_ns=np.int64,
                  count=np.int32)
        a = {k: np.ascontiguousarray(bk[k], dtype=v) for k, v in dt.items()}
        rc = self.lib.oracle_set_book(self.h, _p(a["price"]), _p(a["qty"]), _p(a["oid"]),
                                      _p(a["tid"]), _p(a["time_ns"]), _p(a["count"]))
        if rc != 0:
            raise ValueError("book not in priority order or over capacity")

    def init_from_levels(self, bid_px, bid_qty, ask_px, ask_qty, time_ns=0):
        """Every book from a level snapshot (Sec. 5.1.1): one order per listed
        level, OIDs -9000, -9001, ... (bids best first, then asks); inputs
        int32 [n_books][depth].  Returns the number of sides left empty
        because their levels were out of priority order or over capacity."""
        a = [np.ascontiguousarray(x, dtype=np.int32) for x in (bid_px, bid_qty, ask_px, ask_qty)]
        if any(x.shape != a[0].shape or x.ndim != 2 or x.shape[0] != self.n_books for x in a):
            raise ValueError("level arrays must all be [n_books][depth]")
        return int(self.lib.oracle_init_from_levels(self.h, *[_p(x) for x in a], a[0].shape[1],
                                                    int(time_ns)))

    def levels(self, depth: int):
        shp = (self.n_books, depth)
        bp, bq, ap, aq = (np.empty(shp, np.int32) for _ in range(4))
        self.lib.oracle_get_levels(self.h, depth, _p(bp), _p(bq), _p(ap), _p(aq))
        return bp, bq, ap, aq

    def counters(self):
        out = np.empty((self.n_books, len(COUNTERS)), np.int64)
        self.lib.oracle_get_counters(self.h, _p(out))
        return out

    def resting_qty(self):
        out = np.empty(self.n_books, np.int64)
        self.lib.oracle_get_resting_qty(self.h, _p(out))
        return out


def literal_run(msgs: np.ndarray, offsets: np.ndarray, capacity: int, trade_capacity: int,
                overflow_rule: int = 0):
    """Paper-literal array implementation over whole streams (each book from empty)."""
    lib = _lib(LITERAL_SO)
    vp, i32 = ctypes.c_void_p, ctypes.c_int32
    lib.literal_run.argtypes = [vp, vp, i32, i32, i32, i32] + [vp] * 9
    msgs = np.ascontiguousarray(msgs, dtype=MSG_DTYPE)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    n = len(offsets) - 1
    shp = (n, 2, capacity)
    px, qty, oid, tid = (np.empty(shp, np.int32) for _ in range(4))
    tm = np.empty(shp, np.int64)
    cnt = np.empty((n, 2), np.int32)
    trades = np.empty((n, trade_capacity), TRADE_DTYPE)
    ntr = np.empty(n, np.int64)
    ctr = np.empty((n, lib.literal_n_counters()), np.int64)
    rc = lib.literal_run(_p(msgs) if len(msgs) else None, _p(offsets), n, capacity,
                         trade_capacity, overflow_rule, _p(px), _p(qty), _p(oid), _p(tid),
                         _p(tm), _p(cnt), _p(trades), _p(ntr), _p(ctr))
    if rc != 0:
        raise RuntimeError("literal_run failed (%d)" % rc)
    return dict(price=px, qty=qty, oid=oid, tid=tid, time_ns=tm, count=cnt), trades, ntr, ctr


def messages(rows) -> np.ndarray:
    """Build a message array from (type, side, price, qty, oid, tid, time_ns) tuples."""
    return np.array([tuple(r) for r in rows], dtype=MSG_DTYPE)


class EnvOracle:
    """Execution-environment steps (Sec. 5) over n_envs books, see lob_oracle.cpp."""

    STATE_FIELDS = ["submitted", "executed", "id_counter", "last_ask", "last_time"]

    def __init__(self, n_envs, capacity, trade_capacity, n_steps=400, parent_qty=2000,
                 agent_tid=1_000_000, depth=10, p_init_fallback=10_000, lam=0.0,
                 snapshot_cancels=False, passive_ticks=2, tick_size=1):
        lib = _oracle_lib()
        vp, i32 = ctypes.c_void_p, ctypes.c_int32
        lib.oracle_env_create.restype = vp
        lib.oracle_env_create.argtypes = [i32] * 10 + [ctypes.c_double]
        lib.oracle_env_destroy.argtypes = [vp]
        lib.oracle_env_books.restype = vp
        lib.oracle_env_books.argtypes = [vp]
        lib.oracle_env_step.argtypes = [vp, vp, vp, vp, vp, i32] + [vp] * 6 + [i32, vp]
        lib.oracle_env_observe.argtypes = [vp, vp, i32, vp, vp]
        lib.oracle_env_state.argtypes = [vp, vp, vp]
        self.lib = lib
        self.n, self.depth = n_envs, depth
        self.h = lib.oracle_env_create(n_envs, capacity, trade_capacity, n_steps, parent_qty,
                                       agent_tid, depth, p_init_fallback, passive_ticks,
                                       tick_size, float(lam))
        if not self.h:
            raise ValueError("invalid environment configuration")
        lib.oracle_env_set_snapshot_cancels.argtypes = [vp, i32]
        lib.oracle_env_set_snapshot_cancels(self.h, 1 if snapshot_cancels else 0)
        self.books = Oracle(n_envs, capacity, trade_capacity,
                            _borrow=lib.oracle_env_books(self.h))

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.oracle_env_destroy(h)
            self.h = None

    def step(self, replay, offsets, draws, step, threads=None, l1=False, actions=None):
        """One step; the agent acts from `draws` (uint32 [n]) or, when given,
        from `actions` (float32 [n, 4]: sizes at the far-touch, mid, near-touch
        and passive prices).  With l1=True also returns the level-1 state after
        every data message (int32 [len(replay), 4])."""
        replay = np.ascontiguousarray(replay, dtype=MSG_DTYPE)
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        draws = None if draws is None else np.ascontiguousarray(draws, dtype=np.uint32)
        act = None if actions is None else np.ascontiguousarray(actions, dtype=np.float32)
        if act is not None:
            assert act.shape == (self.n, 4)
        n, d = self.n, self.depth
        reward = np.empty(n, np.float32)
        lv = [np.empty((n, d), np.int32) for _ in range(4)]
        fills = np.empty((n, 2), np.int64)
        tr = np.full((len(replay), 4), -7, np.int32) if l1 else None
        self.lib.oracle_env_step(self.h, _p(replay) if len(replay) else None, _p(offsets),
                                 None if draws is None else _p(draws),
                                 None if act is None else _p(act), step, _p(reward),
                                 *[_p(x) for x in lv], _p(fills),
                                 threads or default_threads(), _p(tr) if l1 and len(replay) else None)
        if l1:
            return reward, tuple(lv), fills, tr
        return reward, tuple(lv), fills

    def state(self):
        out = np.empty((self.n, 5), np.int64)
        p0 = np.empty(self.n, np.float64)
        self.lib.oracle_env_state(self.h, _p(out), _p(p0))
        return out, p0

    def observe(self, l1, msgs_per_step, t_init):
        """Observation after the most recent step (see oracle_env_observe):
        l1 int32 [n, M, 4] (that step's trace), t_init int64 [n]."""
        tr = np.ascontiguousarray(l1, dtype=np.int32).reshape(self.n, msgs_per_step, 4)
        t0 = np.ascontiguousarray(t_init, dtype=np.int64)
        obs = np.empty((self.n, 6 * msgs_per_step + 8), np.float32)
        self.lib.oracle_env_observe(self.h, _p(tr), msgs_per_step, _p(t0), _p(obs))
        return obs
