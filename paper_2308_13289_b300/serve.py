"""Continuous-batching server for order-book simulation episodes.

An episode is a book of a given capacity that advances one step per tick for
its length in steps: a window of data messages is produced for it on the
device (the seeded generator stands in for the market-data feed; the paper
replays fixed-size message windows step by step, Sec. 5.1.1), the window is
applied to the book, and the book's top levels are written -- the serving
counterpart of the batched environments of Sec. 5.

Admission by HBM footprint.  The book of every admitted episode stays resident
in one slot of a per-capacity pool.  A waiting episode is admitted, in arrival
order, as soon as a slot of its capacity is free and its footprint -- book
state, trade log, counters, generator state and its step window -- fits the
HBM budget beside the episodes already running.  Episodes that finish free
their slot and their footprint in the same tick, so later arrivals join a
batch that is already running.

Every tick advances ALL admitted episodes by one step.  Per capacity class,
one call of the library's native tick executor (lob_serve_tick, which keeps
the slots' progress) issues everything: the tick's upload (offsets, slots,
restarts) from a pinned ring, one generator launch that writes the active
slots' windows on the pool's generator stream, then one lob_process_batch
launch that applies them and one lob_get_levels_books launch that reports the
levels of the same slots on the pool's processing stream.  The windows are
double-buffered, so the generator produces tick k+1 while tick k is being
processed; the classes run on their own streams and overlap on the device.
This module keeps admission and the episodes' bookkeeping.

The host runs up to RING ticks ahead of the GPU (finishing times follow from
the step counts, so no tick waits for the previous one).  The latency of an
episode-step is the GPU time of its pool's processing of the tick, from the
moment its window is ready to the moment its levels are written, measured by
events on the processing stream; the generator's time per tick is reported
beside it.  With collect=True (tests) every tick is synchronous, timed on the
host, and the per-step levels and trade counts of every episode are kept.
keep_final=True keeps every episode's final book and counters, captured on the
device in stream order when it finishes (valid in both modes); capture_ids
keeps them for the listed episode ids only (a sample to check at full size).
"""
from __future__ import annotations

import collections
import ctypes
import dataclasses
import math
import time

import numpy as np
import torch

import lobgen

from . import N_COUNTERS, Engine, lib
from ._abi import LobServeDesc

MSG_BYTES = 32
RING = 8  # ticks the host may run ahead of the GPU
GEN_STATE_BYTES = lobgen.STATE_BYTES + lobgen.DEFAULT_POOL * lobgen.POOL_ENTRY_BYTES


@dataclasses.dataclass
class Episode:
    id: int
    capacity: int
    n_steps: int
    msgs_per_step: int
    arrival: float             # seconds (wall clock) or tick index (virtual clock)
    admitted: float = math.nan
    done: float = math.nan


def sample_episodes(rate: float, window: float, seed: int, capacities=(100, 250, 500),
                    steps=(200, 2000), msgs=(100, 500)) -> list:
    """Poisson arrivals at `rate` per second over `window` seconds; capacity,
    length and messages per step drawn uniformly (seeded)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out, t = [], 0.0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= window:
            break
        out.append(Episode(id=len(out), capacity=int(capacities[rng.integers(len(capacities))]),
                           n_steps=int(rng.integers(steps[0], steps[1] + 1)),
                           msgs_per_step=int(rng.integers(msgs[0], msgs[1] + 1)), arrival=t))
    return out


def book_bytes(capacity: int) -> int:
    """Device bytes of one book of this capacity (48 per slot, capacity
    rounded up to a power-of-two multiple of 32 slots)."""
    k = 1
    while 32 * k < capacity:
        k *= 2
    return 48 * 32 * k


def footprint_bytes(capacity: int, trade_capacity: int, msgs_per_step: int) -> int:
    """HBM an admitted episode holds while it runs: its book (state and the two
    side counts), its trade log and count, its counters, its generator state
    and its step window."""
    return (book_bytes(capacity) + 8 + 32 * trade_capacity + 8 + 8 * N_COUNTERS
            + GEN_STATE_BYTES + MSG_BYTES * msgs_per_step)


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


class _Pool:
    """Resident slots of one capacity class: an engine context over all slots,
    per-slot generator state, two window buffers, two streams, and the native
    tick executor (lob_serve_*) that keeps the slots' progress and issues each
    tick."""

    def __init__(self, capacity, slots, trade_capacity, depth, params, max_mps, collect):
        self.capacity, self.slots, self.depth, self.params = capacity, slots, depth, params
        self.max_mps = max_mps
        # processing ahead of window generation when both have blocks waiting
        # for an SM (the step latency is the processing's)
        self.stream = torch.cuda.Stream(priority=-1)  # processing
        self.gstream = torch.cuda.Stream(priority=0)  # window generation
        S = slots
        with torch.cuda.stream(self.stream):
            self.engine = Engine(slots, capacity, trade_capacity, stream=self.stream)
            self.g_states = torch.zeros(S * lobgen.STATE_BYTES, dtype=torch.uint8, device="cuda")
            self.g_pools = torch.zeros(S * params.pool_cap * lobgen.POOL_ENTRY_BYTES,
                                       dtype=torch.uint8, device="cuda")
            self.geo_px = torch.from_numpy(lobgen.GEO_PX.view(np.int64)).cuda()
            self.geo_q = torch.from_numpy(lobgen.GEO_Q.view(np.int64)).cuda()
            self.win = [torch.empty((S * max_mps, 8), dtype=torch.int32, device="cuda")
                        for _ in range(2)]
            self.levels = [torch.empty((S, depth), dtype=torch.int32, device="cuda")
                           for _ in range(4)]
            self.d_tcount = torch.empty(S, dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()
        self.reserved_bytes = (S * (book_bytes(capacity) + 8 + 32 * trade_capacity + 8
                                    + 8 * N_COUNTERS + GEN_STATE_BYTES)
                               + 2 * S * max_mps * MSG_BYTES)
        lg = lobgen.cuda_lib()
        addr = lambda f: ctypes.cast(f, ctypes.c_void_p).value  # noqa: E731
        self.desc = LobServeDesc(
            engine=self.engine.h.value, gen_params=ctypes.addressof(params),
            gen_init=addr(lg.lobgen_dev_init_ids), gen_advance=addr(lg.lobgen_dev_advance),
            d_geo_px=self.geo_px.data_ptr(), d_geo_q=self.geo_q.data_ptr(),
            d_gen_states=self.g_states.data_ptr(), d_gen_pools=self.g_pools.data_ptr(),
            d_win0=self.win[0].data_ptr(), d_win1=self.win[1].data_ptr(),
            d_bid_px=self.levels[0].data_ptr(), d_bid_qty=self.levels[1].data_ptr(),
            d_ask_px=self.levels[2].data_ptr(), d_ask_qty=self.levels[3].data_ptr(),
            d_trade_counts=self.d_tcount.data_ptr(), proc_stream=self.stream.cuda_stream,
            gen_stream=self.gstream.cuda_stream, slots=S, max_msgs=max_mps, depth=depth,
            ring=RING)
        lb = lib()
        self.h = ctypes.c_void_p()
        if lb.lob_serve_create(ctypes.byref(self.h), ctypes.byref(self.desc)) != 0:
            raise RuntimeError("lob_serve_create: %s" % lb.lob_last_error().decode())
        # the executor's outputs of a tick (host buffers reused every tick)
        self.b_act = np.empty(S, np.int32)
        self.b_fin = np.empty(S, np.int32)
        self.b_n = np.zeros(2, np.int32)     # slots advanced, episodes finished
        self.b_msgs = np.zeros(1, np.int64)
        self._tick = lb.lob_serve_tick
        self._tick_args = [None if not collect else ctypes.c_void_p(self.b_act.ctypes.data),
                           ctypes.c_void_p(self.b_n.ctypes.data),
                           ctypes.c_void_p(self.b_fin.ctypes.data),
                           ctypes.c_void_p(self.b_n.ctypes.data + 4),
                           ctypes.c_void_p(self.b_msgs.ctypes.data)]
        self.lat = []      # (GPU ms of a timed tick's processing, episodes in it)
        self.gen_ms = []   # GPU ms of a timed tick's window generation
        self.ep = np.full(slots, -1, np.int64)  # episode index in the slot, -1 free
        self.n_free = slots
        self.n_active = 0
        self.collect = collect

    def flush(self):
        """Wait for every tick issued; collect the timed ticks' times."""
        lb = lib()
        cnt = ctypes.c_int32()
        if lb.lob_serve_timings(self.h, None, None, None, 0, ctypes.byref(cnt)) != 0:
            raise RuntimeError("lob_serve_timings: %s" % lb.lob_last_error().decode())
        n = cnt.value
        if n:
            pm, gm, k = np.empty(n, np.float32), np.empty(n, np.float32), np.empty(n, np.int32)
            if lb.lob_serve_timings(self.h, pm.ctypes.data, gm.ctypes.data, k.ctypes.data, n,
                                    ctypes.byref(cnt)) != 0:
                raise RuntimeError("lob_serve_timings: %s" % lb.lob_last_error().decode())
            self.lat.extend(zip(pm.tolist(), k.tolist()))
            self.gen_ms.extend(gm.tolist())

    def admit(self, idx: int, ep: Episode):
        if ep.msgs_per_step > self.max_mps:
            raise ValueError("episode %d: %d messages per step above the pool's %d"
                             % (ep.id, ep.msgs_per_step, self.max_mps))
        slot = ctypes.c_int32()
        if lib().lob_serve_admit(self.h, ep.id, ep.n_steps, ep.msgs_per_step,
                                 ctypes.byref(slot)) != 0:
            raise RuntimeError("lob_serve_admit: %s" % lib().lob_last_error().decode())
        self.ep[slot.value] = idx
        self.n_free -= 1
        self.n_active += 1

    def launch_step(self, timing=False):
        """One step of every active slot, issued asynchronously by the native
        executor (windows on the generator stream, processing and levels on
        the processing stream).  Returns (active slots -- in collect mode
        only --, messages, slots whose episode ended, episodes advanced)."""
        if self._tick(self.h, 1 if timing else 0, 1 if self.collect else 0, *self._tick_args) != 0:
            raise RuntimeError("lob_serve_tick: %s" % lib().lob_last_error().decode())
        n, nf = int(self.b_n[0]), int(self.b_n[1])
        act = self.b_act[:n].copy() if self.collect else None
        return act, int(self.b_msgs[0]), self.b_fin[:nf].copy(), n

    def ready(self):
        """Whether a tick issued now would not wait for the GPU."""
        r = lib().lob_serve_ready(self.h)
        if r < 0:
            raise RuntimeError("lob_serve_ready: %s" % lib().lob_last_error().decode())
        return r == 1

    def capture_final(self):
        """The pool's books and counters as they stand once the work queued so
        far has run (device tensors, filled in stream order)."""
        with torch.cuda.stream(self.stream):
            bk = self.engine.book()
            ctr, _ = self.engine.stats()
        return bk, ctr

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().lob_serve_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous batching over slot pools with HBM admission: one pool per
    capacity, or, with window_buckets (ascending message counts), one per
    capacity and range of messages per step -- a pool's tick lasts as long
    as its longest window, so episodes with short windows finish their steps
    sooner in a pool of their own."""

    def __init__(self, capacities=(100, 250, 500), hbm_budget=2 << 30, trade_capacity=2048,
                 depth=10, seed=20230829, max_slots=4096, collect=False, keep_final=False,
                 msgs_per_step=(100, 500), capture_ids=None, window_buckets=(),
                 independent=False):
        self.params = lobgen.make_params(seed, "pm1")
        self.depth = depth
        self.budget = hbm_budget
        self.tcap = trade_capacity
        self.collect = collect
        self.keep_final = keep_final or collect
        self.capture_ids = set(capture_ids) if capture_ids else set()
        # independent=True: a loop pass issues a tick only to the pools whose
        # tick would not wait for the GPU, so pools of short windows advance
        # at their own pace instead of the slowest pool's (run-ahead path only)
        self.independent = independent
        lo, hi = msgs_per_step
        # message-count ranges of the pools of one capacity: (lo, b0], (b0, b1], ..., (bk, hi]
        self.bounds = [b for b in sorted(window_buckets) if lo <= b < hi]
        edges = [lo - 1] + self.bounds + [hi]
        self.pools = {}
        for c in capacities:
            for k in range(len(edges) - 1):
                w_lo, w_hi = edges[k] + 1, edges[k + 1]
                # as many slots as the budget holds of the smallest episodes
                slots = int(min(max_slots, max(1, hbm_budget //
                                               footprint_bytes(c, trade_capacity, max(w_lo, 0)))))
                self.pools[(c, k)] = _Pool(c, slots, trade_capacity, depth, self.params, w_hi,
                                           collect)
        self.used = 0
        self.records = collections.defaultdict(list)  # episode id -> per-step outputs
        self.final_books = {}
        self.final_counters = {}

    def footprint(self, ep):
        return footprint_bytes(ep.capacity, self.tcap, ep.msgs_per_step)

    def pool_of(self, ep):
        k = sum(1 for b in self.bounds if ep.msgs_per_step > b)
        return self.pools.get((ep.capacity, k))

    def _admit_waiting(self, episodes, waiting, fps, min_fp, now):
        """First fit in arrival order; stops as soon as no waiting episode
        could fit the budget left, and passes over classes without a free
        slot.  Returns the episodes still waiting."""
        still = collections.deque()
        while waiting:
            if self.used + min_fp > self.budget:
                still.extend(waiting)
                break
            i = waiting.popleft()
            ep = episodes[i]
            pool = self.pool_of(ep)
            if pool is None:
                raise ValueError("no pool for capacity %d" % ep.capacity)
            if pool.n_free and self.used + fps[i] <= self.budget:
                pool.admit(i, ep)
                self.used += fps[i]
                ep.admitted = now
            else:
                still.append(i)
        return still

    def run(self, episodes, clock="wall", max_ticks=None):
        """Serve `episodes` (arrival in seconds for clock='wall', in ticks for
        clock='virtual'); returns a report dict."""
        fps = [self.footprint(ep) for ep in episodes]
        if any(f > self.budget for f in fps):
            raise ValueError("an episode alone exceeds the HBM budget")
        min_fp = min(fps) if fps else 0
        order = sorted(range(len(episodes)), key=lambda i: episodes[i].arrival)
        pending = collections.deque(order)
        waiting = collections.deque()
        lat, weights, queue_len = [], [], []
        finals = []  # (episode id, pool, slot, captured tensors)
        steps_done = msgs_done = 0
        max_active = max_used = 0
        tick = 0
        t0 = time.perf_counter()
        while pending or waiting or any(p.n_active for p in self.pools.values()):
            now = (time.perf_counter() - t0) if clock == "wall" else float(tick)
            while pending and episodes[pending[0]].arrival <= now:
                waiting.append(pending.popleft())
            waiting = self._admit_waiting(episodes, waiting, fps, min_fp, now)
            queue_len.append((now, len(waiting)))
            active = sum(p.n_active for p in self.pools.values())
            max_active = max(max_active, active)
            max_used = max(max_used, self.used)
            busy = [p for p in self.pools.values() if p.n_active]
            if not busy:
                if clock == "wall" and pending:
                    time.sleep(max(0.0, min(episodes[pending[0]].arrival - now, 0.001)))
                tick += 1
                continue
            if self.collect:
                ts = time.perf_counter()
                launched = [(p, *p.launch_step()) for p in busy]
                for p in busy:
                    p.stream.synchronize()
                te = time.perf_counter()
                lat.append(te - ts)
                weights.append(active)
                self._record(episodes, launched)
            else:
                te = time.perf_counter()
                if self.independent:
                    busy = [p for p in busy if p.ready()]
                    if not busy:  # every pool's next tick would wait: let the GPU catch up
                        time.sleep(0)
                        continue
                launched = [(p, *p.launch_step(timing=True)) for p in busy]
            steps_done += sum(n for *_, n in launched)
            msgs_done += sum(m for _, _, m, _, _ in launched)
            now_after = (te - t0) if clock == "wall" else float(tick)
            for p, _, _, ended, _ in launched:
                if not len(ended):
                    continue
                keep = [s for s in ended if self.keep_final or
                        episodes[int(p.ep[s])].id in self.capture_ids]
                if keep:
                    cap = p.capture_final()
                    for s in keep:
                        finals.append((episodes[int(p.ep[s])].id, int(s), cap))
                for s in ended:
                    i = int(p.ep[s])
                    episodes[i].done = now_after
                    p.ep[s] = -1
                    p.n_active -= 1
                    p.n_free += 1
                    self.used -= fps[i]
            tick += 1
            if max_ticks is not None and tick >= max_ticks:
                break
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        gen_ms = []
        per_pool = {}
        by_cap = collections.defaultdict(list)
        for (c, _), p in self.pools.items():
            p.flush()
            by_cap[c] += p.lat
        for c, pl in by_cap.items():
            if pl:
                pl = np.repeat(np.asarray([ms for ms, _ in pl]), [n for _, n in pl])
                per_pool[c] = {"p50_step_ms": float(np.percentile(pl, 50)),
                               "p99_step_ms": float(np.percentile(pl, 99)),
                               "episode_steps": int(len(pl))}
        for p in self.pools.values():
            for ms, n in p.lat:
                lat.append(ms / 1e3)
                weights.append(n)
            gen_ms += p.gen_ms
            p.lat, p.gen_ms = [], []
        for eid, s, (bk, ctr) in finals:
            self.final_books[eid] = {k: v[s].cpu().numpy().copy() for k, v in bk.items()}
            self.final_counters[eid] = ctr[s].cpu().numpy().copy()
        lat_ms = np.repeat(np.asarray(lat) * 1e3, weights) if lat else np.zeros(1)
        waits = [e.admitted - e.arrival for e in episodes if not math.isnan(e.admitted)]
        return {"episodes": len(episodes), "episode_steps": steps_done, "messages": msgs_done,
                "wall_s": wall, "ticks": tick,
                "steps_per_s": steps_done / wall, "msgs_per_s": msgs_done / wall,
                "p50_step_ms": float(np.percentile(lat_ms, 50)),
                "p99_step_ms": float(np.percentile(lat_ms, 99)),
                "p50_window_gen_ms": float(np.percentile(gen_ms, 50)) if gen_ms else None,
                "mean_batch": float(np.mean(weights)) if weights else 0.0,
                "admission_wait_p50": float(np.percentile(waits, 50)) if waits else 0.0,
                "admission_wait_p99": float(np.percentile(waits, 99)) if waits else 0.0,
                "max_queue": max(q for _, q in queue_len) if queue_len else 0,
                "max_active": max_active, "max_hbm_bytes_admitted": max_used,
                "hbm_budget_bytes": self.budget,
                "hbm_reserved_bytes": sum(p.reserved_bytes for p in self.pools.values()),
                "slots": {("%d" % c if not self.bounds else "%d/%d" % (c, k)): p.slots
                          for (c, k), p in self.pools.items()},
                "window_buckets": list(self.bounds),
                "per_capacity": per_pool,
                "queue": queue_len}

    def _record(self, episodes, launched):
        for p, act, _, _, _ in launched:
            lv = [x.cpu().numpy() for x in p.levels]
            tc = p.d_tcount.cpu().numpy()
            for s in act:
                ep = episodes[int(p.ep[s])]
                self.records[ep.id].append((tuple(x[s].tolist() for x in lv), int(tc[s])))
