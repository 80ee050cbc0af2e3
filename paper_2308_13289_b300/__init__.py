"""Batched price-time-priority limit-order-book engine for B300 (sm_103a).

Thin binding over ``liblob.so`` (C ABI in ``include/lob.h``): every step of the
path runs in the library's CUDA kernels; this module only marshals torch CUDA
tensors (device memory) and the current torch stream into the calls.

Record layouts on the device (torch ``int32`` tensors, 8 words per record):
  message  [type, side, price, qty, oid, tid, time_lo, time_hi]   (Sec. 4.2)
  trade    [price, qty, oid_aggr, oid_stand, tid_aggr, tid_stand, time_lo, time_hi]
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _abi
from ._abi import LobConfig, LobEnvConfig, LobError, check

OVERFLOW_EVICT, OVERFLOW_REJECT = 0, 1
FLAG_APPEND_TRADES = 1
FLAG_SNAPSHOT_CANCELS = 2
N_COUNTERS = 20
COUNTERS = ["msgs", "limit", "cancel", "market", "noop", "invalid", "trades", "traded_qty",
            "rested", "rejected", "rejected_qty", "evicted", "evicted_qty", "cancel_hit",
            "cancelled_qty", "cancel_miss", "market_discarded_qty", "limit_qty", "market_qty",
            "trades_dropped"]
STATUS_TIMEOUT, STATUS_BAD_BOOK, STATUS_BAD_SEGMENT, STATUS_BAD_BOOK_LOAD = 1, 2, 4, 8
STATUS_CHECK = 16  # checked builds only

MSG_DTYPE = np.dtype([("type", "<i4"), ("side", "<i4"), ("price", "<i4"), ("qty", "<i4"),
                      ("oid", "<i4"), ("tid", "<i4"), ("time_ns", "<i8")])
TRADE_DTYPE = np.dtype([("price", "<i4"), ("qty", "<i4"), ("oid_aggr", "<i4"),
                        ("oid_stand", "<i4"), ("tid_aggr", "<i4"), ("tid_stand", "<i4"),
                        ("time_ns", "<i8")])


def lib():
    return _abi.load()


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def messages_to_device(msgs: np.ndarray, device="cuda") -> torch.Tensor:
    """numpy message records (32 B each) -> int32 [N, 8] CUDA tensor."""
    a = np.ascontiguousarray(msgs).view(np.int32).reshape(-1, 8)
    return torch.from_numpy(a).to(device)


def trades_to_numpy(t: torch.Tensor) -> np.ndarray:
    """int32 [..., 8] trade tensor -> numpy structured records."""
    a = np.ascontiguousarray(t.cpu().numpy())
    return a.view(TRADE_DTYPE).reshape(a.shape[:-1])


# ------------------------------------------------------------------ raw C ABI (same names)

def lob_create(n_books, capacity, trade_capacity, overflow_rule=0, flags=0, stream=None):
    h = ctypes.c_void_p()
    cfg = LobConfig(n_books, capacity, trade_capacity, overflow_rule, flags)
    check(lib().lob_create(ctypes.byref(h), ctypes.byref(cfg), _stream(stream)), "lob_create")
    return h


def lob_destroy(h):
    check(lib().lob_destroy(h), "lob_destroy")


def lob_reset(h, stream=None):
    check(lib().lob_reset(h, _stream(stream)), "lob_reset")


def lob_reset_books(h, book_ids, stream=None):
    check(lib().lob_reset_books(h, _ptr(book_ids), book_ids.numel(), _stream(stream)),
          "lob_reset_books")


def lob_process_batch(h, msgs, offsets, book_ids=None, n_active=None, stream=None):
    n = (offsets.numel() - 1) if n_active is None else n_active
    check(lib().lob_process_batch(h, _ptr(msgs), _ptr(offsets), _ptr(book_ids), n,
                                  _stream(stream)), "lob_process_batch")


def lob_process_batch_l1(h, msgs, offsets, l1, book_ids=None, n_active=None, stream=None):
    n = (offsets.numel() - 1) if n_active is None else n_active
    check(lib().lob_process_batch_l1(h, _ptr(msgs), _ptr(offsets), _ptr(book_ids), n, _ptr(l1),
                                     _stream(stream)), "lob_process_batch_l1")


def lob_process_segments(h, msgs, starts, counts, book_ids, stream=None):
    check(lib().lob_process_segments(h, _ptr(msgs), _ptr(starts), _ptr(counts), _ptr(book_ids),
                                     book_ids.numel(), _stream(stream)), "lob_process_segments")


def _host_ptr(t):
    if t.is_cuda:
        raise ValueError("expected a host tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def lob_selftest_wait(limit_ns, status, elapsed=None, stream=None):
    check(lib().lob_selftest_wait(int(limit_ns), _ptr(status), _ptr(elapsed), _stream(stream)),
          "lob_selftest_wait")


def lob_process_host(h, h_msgs, msgs_per_book, chunk_msgs, stream=None):
    check(lib().lob_process_host(h, _host_ptr(h_msgs), int(msgs_per_book), int(chunk_msgs),
                                 _stream(stream)), "lob_process_host")


def lob_inject_orders(h, msgs, offsets, book_ids=None, n_active=None, stream=None):
    n = (offsets.numel() - 1) if n_active is None else n_active
    check(lib().lob_inject_orders(h, _ptr(msgs), _ptr(offsets), _ptr(book_ids), n,
                                  _stream(stream)), "lob_inject_orders")


def lob_clear_trades(h, stream=None):
    check(lib().lob_clear_trades(h, _stream(stream)), "lob_clear_trades")


def lob_get_levels(h, depth, bid_px, bid_qty, ask_px, ask_qty, stream=None):
    check(lib().lob_get_levels(h, depth, _ptr(bid_px), _ptr(bid_qty), _ptr(ask_px),
                               _ptr(ask_qty), _stream(stream)), "lob_get_levels")


def lob_get_levels_books(h, book_ids, n_active, depth, bid_px, bid_qty, ask_px, ask_qty,
                         stream=None):
    check(lib().lob_get_levels_books(h, _ptr(book_ids), n_active, depth, _ptr(bid_px),
                                     _ptr(bid_qty), _ptr(ask_px), _ptr(ask_qty),
                                     _stream(stream)), "lob_get_levels_books")


def lob_get_trades(h, out, counts, stream=None):
    check(lib().lob_get_trades(h, _ptr(out), _ptr(counts), _stream(stream)), "lob_get_trades")


def lob_get_book(h, px, qty, oid, tid, tm, count, stream=None):
    check(lib().lob_get_book(h, _ptr(px), _ptr(qty), _ptr(oid), _ptr(tid), _ptr(tm),
                             _ptr(count), _stream(stream)), "lob_get_book")


def lob_set_book(h, px, qty, oid, tid, tm, count, stream=None):
    check(lib().lob_set_book(h, _ptr(px), _ptr(qty), _ptr(oid), _ptr(tid), _ptr(tm),
                             _ptr(count), _stream(stream)), "lob_set_book")


def lob_init_from_levels(h, bid_px, bid_qty, ask_px, ask_qty, time_ns=0, stream=None):
    depth = bid_px.shape[-1]
    for t in (bid_qty, ask_px, ask_qty):
        if t.shape != bid_px.shape or t.dtype != torch.int32:
            raise ValueError("level arrays must be int32 tensors of one shape [n_books, depth]")
    check(lib().lob_init_from_levels(h, _ptr(bid_px), _ptr(bid_qty), _ptr(ask_px), _ptr(ask_qty),
                                     int(depth), int(time_ns), _stream(stream)),
          "lob_init_from_levels")


def lob_get_stats(h, counters, status, stream=None):
    check(lib().lob_get_stats(h, _ptr(counters), _ptr(status), _stream(stream)), "lob_get_stats")


def lob_set_launch(h, warps_per_cta, chunk_msgs, ctas_per_sm=0):
    check(lib().lob_set_launch(h, warps_per_cta, chunk_msgs, ctas_per_sm), "lob_set_launch")


def lob_launch_count(h):
    return int(lib().lob_launch_count(h))


def lob_process_streams_static(msgs, offsets, n_books, capacity, trade_capacity, overflow_rule,
                               trades, trade_counts, counters, px=None, qty=None, oid=None,
                               tid=None, tm=None, count=None, status=None, stream=None):
    """Allocation-free variant (no context; books start empty; fixed scratch
    inside the library).  All outputs are caller-owned CUDA tensors."""
    check(lib().lob_process_streams_static(
        _ptr(msgs), _ptr(offsets), n_books, capacity, trade_capacity, overflow_rule,
        _ptr(trades), _ptr(trade_counts), _ptr(counters), _ptr(px), _ptr(qty), _ptr(oid),
        _ptr(tid), _ptr(tm), _ptr(count), _ptr(status), _stream(stream)),
        "lob_process_streams_static")


def lob_env_create(h, n_steps, parent_qty, agent_tid, depth, p_init_fallback, msgs_per_step,
                   lam=0.0, passive_ticks=2, tick_size=1, stream=None):
    e = ctypes.c_void_p()
    cfg = LobEnvConfig(n_steps, parent_qty, agent_tid, depth, p_init_fallback, msgs_per_step,
                       float(lam), passive_ticks, tick_size)
    check(lib().lob_env_create(ctypes.byref(e), h, ctypes.byref(cfg), _stream(stream)),
          "lob_env_create")
    return e


def lob_env_destroy(e):
    check(lib().lob_env_destroy(e), "lob_env_destroy")


def lob_env_reset(e, stream=None):
    check(lib().lob_env_reset(e, _stream(stream)), "lob_env_reset")


def lob_env_run(e, replay, stride_env, step0, n_run, draws, reward, bid_px, bid_qty, ask_px,
                ask_qty, fills, l1=None, actions=None, stream=None):
    check(lib().lob_env_run(e, _ptr(replay), stride_env, step0, n_run, _ptr(draws),
                            _ptr(actions), _ptr(reward), _ptr(bid_px), _ptr(bid_qty),
                            _ptr(ask_px), _ptr(ask_qty), _ptr(fills), _ptr(l1), _stream(stream)),
          "lob_env_run")


def lob_env_observe(e, replay, stride_env, l1, obs, stream=None):
    check(lib().lob_env_observe(e, _ptr(replay), stride_env, _ptr(l1), _ptr(obs),
                                _stream(stream)), "lob_env_observe")


def lob_env_segments(e):
    return int(lib().lob_env_segments(e))


def lob_env_get_state(e, state, p_init, stream=None):
    check(lib().lob_env_get_state(e, _ptr(state), _ptr(p_init), _stream(stream)),
          "lob_env_get_state")


def lob_literal_process(msgs, offsets, n_books, capacity, trade_capacity, overflow_rule,
                        all_branches, trades, trade_counts, px, qty, oid, tid, tm, count,
                        stream=None):
    check(lib().lob_literal_process(_ptr(msgs), _ptr(offsets), n_books, capacity,
                                    trade_capacity, overflow_rule, int(all_branches),
                                    _ptr(trades), _ptr(trade_counts), _ptr(px), _ptr(qty),
                                    _ptr(oid), _ptr(tid), _ptr(tm), _ptr(count),
                                    _stream(stream)), "lob_literal_process")


def literal_process(msgs, offsets, capacity, trade_capacity, overflow_rule=OVERFLOW_EVICT,
                    all_branches=True, stream=None):
    """The paper-literal ablation (lob_literal_process): every book from empty
    over its segment.  Returns (book dict in the Engine.book() layout, trades
    [n, trade_capacity, 8] int32 view, trade counts)."""
    n = offsets.numel() - 1
    shape = (n, 2, capacity)
    bk = {k: torch.empty(shape, dtype=torch.int32, device="cuda")
          for k in ("price", "qty", "oid", "tid")}
    bk["time_ns"] = torch.empty(shape, dtype=torch.int64, device="cuda")
    bk["count"] = torch.empty((n, 2), dtype=torch.int32, device="cuda")
    tr = torch.empty((n, max(1, trade_capacity), 8), dtype=torch.int32, device="cuda")
    cnt = torch.empty(n, dtype=torch.int64, device="cuda")
    lob_literal_process(msgs, offsets, n, capacity, trade_capacity, overflow_rule, all_branches,
                        tr, cnt, bk["price"], bk["qty"], bk["oid"], bk["tid"], bk["time_ns"],
                        bk["count"], stream)
    return bk, tr[:, :trade_capacity], cnt


# ------------------------------------------------------------------ convenience object

class Engine:
    """A lob_ctx with torch-allocated outputs.  All calls run on the current
    torch stream unless `stream` is given."""

    def __init__(self, n_books: int, capacity: int, trade_capacity: int,
                 overflow_rule: int = OVERFLOW_EVICT, append_trades: bool = False,
                 snapshot_cancels: bool = False, stream=None):
        self.n_books, self.capacity, self.trade_capacity = n_books, capacity, trade_capacity
        self.stream = stream
        flags = (FLAG_APPEND_TRADES if append_trades else 0) | \
                (FLAG_SNAPSHOT_CANCELS if snapshot_cancels else 0)
        self.h = lob_create(n_books, capacity, trade_capacity, overflow_rule, flags, stream)

    def close(self):
        if getattr(self, "h", None):
            lob_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self):
        lob_reset(self.h, self.stream)

    def reset_books(self, book_ids):
        lob_reset_books(self.h, book_ids, self.stream)

    def process_batch(self, msgs, offsets, book_ids=None):
        lob_process_batch(self.h, msgs, offsets, book_ids, stream=self.stream)

    def process_host(self, h_msgs, msgs_per_book, chunk_msgs=2000):
        """Every book's messages from pinned host memory (book-major, equal
        counts), copied chunk by chunk while the previous chunk is processed."""
        lob_process_host(self.h, h_msgs, msgs_per_book, chunk_msgs, self.stream)

    def inject_orders(self, msgs, offsets, book_ids=None):
        lob_inject_orders(self.h, msgs, offsets, book_ids, stream=self.stream)

    def clear_trades(self):
        lob_clear_trades(self.h, self.stream)

    def set_launch(self, warps_per_cta, chunk_msgs, ctas_per_sm=0):
        lob_set_launch(self.h, warps_per_cta, chunk_msgs, ctas_per_sm)

    def launch_count(self):
        return lob_launch_count(self.h)

    def levels(self, depth: int):
        out = [torch.empty((self.n_books, depth), dtype=torch.int32, device="cuda")
               for _ in range(4)]
        lob_get_levels(self.h, depth, *out, stream=self.stream)
        return tuple(out)

    def levels_of(self, book_ids, depth: int, out=None):
        """Levels of the listed books (int32 CUDA tensor of ids) written to
        their rows of `out` (four int32 [n_books, depth] tensors, allocated
        filled with -7 when None); other rows are left as they are."""
        if out is None:
            out = [torch.full((self.n_books, depth), -7, dtype=torch.int32, device="cuda")
                   for _ in range(4)]
        lob_get_levels_books(self.h, book_ids, int(book_ids.numel()), depth, *out,
                             stream=self.stream)
        return tuple(out)

    def trades(self):
        out = torch.empty((self.n_books, max(self.trade_capacity, 0), 8), dtype=torch.int32,
                          device="cuda")
        cnt = torch.empty(self.n_books, dtype=torch.int64, device="cuda")
        lob_get_trades(self.h, out if self.trade_capacity > 0 else None, cnt, self.stream)
        return out, cnt

    def book(self):
        shp = (self.n_books, 2, self.capacity)
        px, qty, oid, tid = (torch.empty(shp, dtype=torch.int32, device="cuda")
                             for _ in range(4))
        tm = torch.empty(shp, dtype=torch.int64, device="cuda")
        cnt = torch.empty((self.n_books, 2), dtype=torch.int32, device="cuda")
        lob_get_book(self.h, px, qty, oid, tid, tm, cnt, self.stream)
        return dict(price=px, qty=qty, oid=oid, tid=tid, time_ns=tm, count=cnt)

    def set_book(self, bk: dict):
        t = {k: bk[k].contiguous() for k in ("price", "qty", "oid", "tid", "time_ns", "count")}
        lob_set_book(self.h, t["price"], t["qty"], t["oid"], t["tid"], t["time_ns"], t["count"],
                     self.stream)

    def init_from_levels(self, bid_px, bid_qty, ask_px, ask_qty, time_ns=0):
        """Every book from a level snapshot (lob_init_from_levels, Sec. 5.1.1):
        int32 CUDA tensors [n_books, depth] in the lob_get_levels layout."""
        if bid_px.dim() != 2 or bid_px.shape[0] != self.n_books:
            raise ValueError("level arrays must be [n_books, depth]")
        t = [x.contiguous() for x in (bid_px, bid_qty, ask_px, ask_qty)]
        lob_init_from_levels(self.h, *t, time_ns=time_ns, stream=self.stream)

    def stats(self):
        ctr = torch.empty((self.n_books, N_COUNTERS), dtype=torch.int64, device="cuda")
        st = torch.empty(1, dtype=torch.int32, device="cuda")
        lob_get_stats(self.h, ctr, st, self.stream)
        return ctr, st


class Env:
    """Execution environments over the books of an Engine (see lob_env_* in lob.h)."""

    def __init__(self, engine: "Engine", n_steps=400, parent_qty=2000, agent_tid=1_000_000,
                 depth=10, p_init_fallback=10_000, msgs_per_step=100, lam=0.0, passive_ticks=2,
                 tick_size=1, stream=None):
        self.engine, self.n, self.depth, self.stream = engine, engine.n_books, depth, stream
        self.n_steps, self.msgs_per_step = n_steps, msgs_per_step
        self.h = lob_env_create(engine.h, n_steps, parent_qty, agent_tid, depth, p_init_fallback,
                                msgs_per_step, lam, passive_ticks, tick_size, stream)

    def close(self):
        if getattr(self, "h", None):
            lob_env_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self):
        lob_env_reset(self.h, self.stream)

    def outputs(self, n_run):
        n, d = self.n, self.depth
        return dict(reward=torch.empty((n_run, n), dtype=torch.float32, device="cuda"),
                    bid_px=torch.empty((n_run, n, d), dtype=torch.int32, device="cuda"),
                    bid_qty=torch.empty((n_run, n, d), dtype=torch.int32, device="cuda"),
                    ask_px=torch.empty((n_run, n, d), dtype=torch.int32, device="cuda"),
                    ask_qty=torch.empty((n_run, n, d), dtype=torch.int32, device="cuda"),
                    fills=torch.empty((n_run, n, 2), dtype=torch.int64, device="cuda"))

    def run(self, replay, stride_env, step0, n_run, draws, out=None, row0=0, l1=None,
            actions=None):
        """Steps step0..step0+n_run-1; the agent acts from draws (int32/uint32
        [n_run, n], the seeded stand-in) or, with draws=None, from actions
        (float32 [n_run, n, 4], sizes at the far-touch, mid, near-touch and
        passive prices); results go to rows row0.. of `out` (allocated when
        None); l1: optional int32 [n_run, n, msgs_per_step, 4] level-1 trace of
        the data messages."""
        if out is None:
            out = self.outputs(n_run)
            row0 = 0
        sl = {k: v[row0:row0 + n_run] for k, v in out.items()}
        lob_env_run(self.h, replay, stride_env, step0, n_run, draws, sl["reward"], sl["bid_px"],
                    sl["bid_qty"], sl["ask_px"], sl["ask_qty"], sl["fills"], l1, actions,
                    self.stream)
        return out

    def observe(self, replay, stride_env, l1, obs=None):
        """Observation after the most recent step, float32 [n, 6M + 8]; l1 is
        that step's trace, int32 [n, msgs_per_step, 4]."""
        if obs is None:
            obs = torch.empty((self.n, 6 * self.msgs_per_step + 8), dtype=torch.float32,
                              device="cuda")
        lob_env_observe(self.h, replay, stride_env, l1, obs, self.stream)
        return obs

    def segments(self):
        """Segments per environment of the most recent run (lob_env_segments)."""
        return lob_env_segments(self.h)

    def state(self):
        st = torch.empty((self.n, 5), dtype=torch.int64, device="cuda")
        p0 = torch.empty(self.n, dtype=torch.float64, device="cuda")
        lob_env_get_state(self.h, st, p0, self.stream)
        return st, p0


__all__ = [n for n in dir() if n.startswith("lob_")] + [
    "Engine", "Env", "LobError", "messages_to_device", "trades_to_numpy", "MSG_DTYPE", "TRADE_DTYPE",
    "COUNTERS", "N_COUNTERS"]
