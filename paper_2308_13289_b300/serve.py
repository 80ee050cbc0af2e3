"""Continuous-batching server for order-book simulation episodes.

An episode is a book of a given capacity that advances one step (a window of
data messages, then its top levels) per tick for its length in steps, the
serving counterpart of the batched environments of Sec. 5.  Episodes arrive
over time; the server keeps the book of every admitted episode resident in
HBM (one slot of a per-capacity pool), admits a waiting episode as soon as a
slot of its capacity is free and its HBM footprint fits the budget, and on
every tick advances ALL admitted episodes by one step: per capacity class one
batched launch over the active slots, each class on its own CUDA stream so
the classes overlap on the device.  Episodes that finish free their slot in
the same tick, so arrivals join a batch that is already running.

Latency of an episode-step = wall time of the tick that ran it; the report
gives p50/p99 over all episode-steps, steps/s and messages/s, the admission
wait and the queue length over time.
"""
from __future__ import annotations

import collections
import ctypes
import dataclasses
import math
import time

import numpy as np
import torch

from . import Engine, lib, lob_get_levels

MSG_BYTES = 32


@dataclasses.dataclass
class Episode:
    id: int
    capacity: int
    n_steps: int
    msgs_per_step: int
    arrival: float             # seconds (wall clock) or tick index (virtual clock)
    slot: int = -1
    step: int = 0
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


def footprint_bytes(capacity: int, trade_capacity: int, max_msgs: int, pool_cap: int) -> int:
    """HBM an admitted episode holds: book state, trade log, generator state
    and its share of the step message buffer."""
    k = 1
    while 32 * k < capacity:
        k *= 2
    return 48 * 32 * k + 32 * trade_capacity + 40 + 16 * pool_cap + MSG_BYTES * max_msgs + 64


class _Pool:
    """Resident slots of one capacity class."""

    def __init__(self, capacity, slots, trade_capacity, depth, params, max_msgs, collect):
        import lobgen
        self.capacity, self.slots, self.depth = capacity, slots, depth
        self.stream = torch.cuda.Stream()
        with torch.cuda.stream(self.stream):
            self.engine = Engine(slots, capacity, trade_capacity, stream=self.stream)
            self.gen = lobgen.DeviceStreams(params, slots)
            self.d_msgs = torch.empty((slots * max_msgs, 8), dtype=torch.int32, device="cuda")
            self.d_off = torch.empty(slots + 1, dtype=torch.int64, device="cuda")
            self.d_ids = torch.empty(slots, dtype=torch.int32, device="cuda")
            self.d_cnt = torch.empty(slots, dtype=torch.int64, device="cuda")
            self.levels = [torch.empty((slots, depth), dtype=torch.int32, device="cuda")
                           for _ in range(4)]
            self.d_tcount = torch.empty(slots, dtype=torch.int64, device="cuda")
        self.h_off = torch.empty(slots + 1, dtype=torch.int64).pin_memory()
        self.h_ids = torch.empty(slots, dtype=torch.int32).pin_memory()
        self.h_cnt = torch.empty(slots, dtype=torch.int64).pin_memory()
        self.free = list(range(slots - 1, -1, -1))
        self.active = {}
        self.collect = collect
        self.lobgen = lobgen
        self.params = params

    def admit(self, ep: Episode):
        ep.slot = self.free.pop()
        self.active[ep.slot] = ep
        with torch.cuda.stream(self.stream):
            ids = torch.tensor([ep.slot], dtype=torch.int32, device="cuda")
            self.engine.reset_books(ids)
            self.gen.restart([ep.slot], [ep.id])

    def launch_step(self):
        """Generate and process one step of every active episode (async)."""
        slots = sorted(self.active)
        n = len(slots)
        counts = np.fromiter((self.active[s].msgs_per_step for s in slots), np.int64, n)
        off = np.zeros(n + 1, np.int64)
        np.cumsum(counts, out=off[1:])
        self.h_ids[:n] = torch.from_numpy(np.asarray(slots, np.int32))
        self.h_cnt[:n] = torch.from_numpy(counts)
        self.h_off[:n + 1] = torch.from_numpy(off)
        glib = self.gen.lib
        s = ctypes.c_void_p(self.stream.cuda_stream)
        with torch.cuda.stream(self.stream):
            self.d_ids[:n].copy_(self.h_ids[:n], non_blocking=True)
            self.d_cnt[:n].copy_(self.h_cnt[:n], non_blocking=True)
            self.d_off[:n + 1].copy_(self.h_off[:n + 1], non_blocking=True)
            p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
            rc = glib.lobgen_dev_advance(ctypes.byref(self.params), p(self.gen.geo_px),
                                         p(self.gen.geo_q), n, p(self.d_ids), p(self.gen.states),
                                         p(self.gen.pools), p(self.d_cnt), p(self.d_off),
                                         p(self.d_msgs), s)
            if rc != 0:
                raise RuntimeError("generator launch failed")
            rc = lib().lob_process_batch(self.engine.h, p(self.d_msgs), p(self.d_off),
                                         p(self.d_ids), n, s)
            if rc != 0:
                raise RuntimeError("lob_process_batch failed")
            lob_get_levels(self.engine.h, self.depth, *self.levels, stream=self.stream)
            if self.collect:
                rc = lib().lob_get_trades(self.engine.h, None, p(self.d_tcount), s)
        return slots, int(off[-1])


class Server:
    """Continuous batching over per-capacity slot pools with HBM admission."""

    def __init__(self, capacities=(100, 250, 500), hbm_budget=2 << 30, trade_capacity=2048,
                 depth=10, max_msgs=500, seed=20230829, max_slots=4096, collect=False):
        import lobgen
        self.params = lobgen.make_params(seed, "pm1")
        self.trade_capacity, self.depth, self.max_msgs = trade_capacity, depth, max_msgs
        self.budget = hbm_budget
        self.fp = {c: footprint_bytes(c, trade_capacity, max_msgs, self.params.pool_cap)
                   for c in capacities}
        self.pools = {c: _Pool(c, min(max_slots, max(1, hbm_budget // self.fp[c])),
                               trade_capacity, depth, self.params, max_msgs, collect)
                      for c in capacities}
        self.used = 0
        self.collect = collect
        self.records = collections.defaultdict(list)  # episode id -> per-step outputs
        self.final_books = {}

    def _can_admit(self, ep):
        pool = self.pools.get(ep.capacity)
        if pool is None:
            raise ValueError("no pool for capacity %d" % ep.capacity)
        if ep.msgs_per_step > self.max_msgs:
            raise ValueError("episode %d has %d messages per step (max %d)"
                             % (ep.id, ep.msgs_per_step, self.max_msgs))
        return bool(pool.free) and self.used + self.fp[ep.capacity] <= self.budget

    def run(self, episodes, clock="wall", max_ticks=None):
        """Serve `episodes` (arrival in seconds for clock='wall', in ticks for
        clock='virtual'); returns a report dict."""
        pending = collections.deque(sorted(episodes, key=lambda e: e.arrival))
        waiting = []
        lat, weights, queue_len = [], [], []
        steps_done = msgs_done = 0
        max_active = max_used = 0
        tick = 0
        t0 = time.perf_counter()
        while pending or waiting or any(p.active for p in self.pools.values()):
            now = (time.perf_counter() - t0) if clock == "wall" else float(tick)
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            still = []
            for ep in waiting:  # first fit, in arrival order
                if self._can_admit(ep):
                    self.pools[ep.capacity].admit(ep)
                    self.used += self.fp[ep.capacity]
                    ep.admitted = now
                else:
                    still.append(ep)
            waiting = still
            queue_len.append((now, len(waiting)))
            max_active = max(max_active, sum(len(p.active) for p in self.pools.values()))
            max_used = max(max_used, self.used)
            busy = [p for p in self.pools.values() if p.active]
            if not busy:
                if clock == "wall" and pending:
                    time.sleep(max(0.0, min(pending[0].arrival - now, 0.001)))
                tick += 1
                continue
            ts = time.perf_counter()
            launched = [(p, *p.launch_step()) for p in busy]
            for p in busy:
                p.stream.synchronize()
            te = time.perf_counter()
            n_eps = sum(len(sl) for _, sl, _ in launched)
            lat.append(te - ts)
            weights.append(n_eps)
            steps_done += n_eps
            msgs_done += sum(m for _, _, m in launched)
            if self.collect:
                self._record(launched)
            now_after = (te - t0) if clock == "wall" else float(tick)
            for p, slots, _ in launched:
                for s in slots:
                    ep = p.active[s]
                    ep.step += 1
                    if ep.step >= ep.n_steps:
                        if self.collect:
                            self._final_book(p, ep)
                        ep.done = now_after
                        del p.active[s]
                        p.free.append(s)
                        self.used -= self.fp[ep.capacity]
            tick += 1
            if max_ticks is not None and tick >= max_ticks:
                break
        wall = time.perf_counter() - t0
        lat_ms = np.repeat(np.asarray(lat) * 1e3, weights) if lat else np.zeros(1)
        waits = [e.admitted - e.arrival for e in episodes if not math.isnan(e.admitted)]
        return {"episodes": len(episodes), "episode_steps": steps_done, "messages": msgs_done,
                "wall_s": wall, "ticks": tick,
                "steps_per_s": steps_done / wall, "msgs_per_s": msgs_done / wall,
                "p50_step_ms": float(np.percentile(lat_ms, 50)),
                "p99_step_ms": float(np.percentile(lat_ms, 99)),
                "mean_batch": float(np.mean(weights)) if weights else 0.0,
                "admission_wait_p50": float(np.percentile(waits, 50)) if waits else 0.0,
                "admission_wait_p99": float(np.percentile(waits, 99)) if waits else 0.0,
                "max_queue": max(q for _, q in queue_len) if queue_len else 0,
                "max_active": max_active, "max_hbm_bytes_admitted": max_used,
                "queue": queue_len}

    def _record(self, launched):
        for p, slots, _ in launched:
            lv = [x.cpu().numpy() for x in p.levels]
            tc = p.d_tcount.cpu().numpy()
            for s in slots:
                ep = p.active[s]
                self.records[ep.id].append((tuple(x[s].tolist() for x in lv), int(tc[s])))

    def _final_book(self, p, ep):
        bk = p.engine.book()
        p.stream.synchronize()
        self.final_books[ep.id] = {k: v[ep.slot].cpu().numpy().copy() for k, v in bk.items()}
