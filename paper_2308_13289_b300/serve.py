"""Continuous-batching server for order-book simulation episodes.

An episode is a book of a given capacity that advances one step (a window of
data messages, then its top levels) per tick for its length in steps -- the
serving counterpart of the batched environments of Sec. 5.  Its message
windows are loaded into HBM when the request is accepted (the paper likewise
pre-loads fixed-size message windows, Sec. 5.1.1).  The server keeps the book
of every admitted episode resident (one slot of a per-capacity pool), admits a
waiting episode as soon as a slot of its capacity is free and its resident
footprint fits the HBM budget, and on every tick advances ALL admitted
episodes by one step: per capacity class one launch over the active slots'
current windows (lob_process_segments), each class on its own CUDA stream so
the classes overlap on the device.  Episodes that finish free their slot in
the same tick, so later arrivals join a batch that is already running.

The host runs up to RING ticks ahead of the GPU (finishing times are known
from the step counts, so no tick waits for the previous one); the latency of
an episode-step is the GPU time of its pool's tick, measured by events around
that tick's work on the pool's stream.  The report gives p50/p99 over all
episode-steps, steps/s and messages/s, the admission wait and the queue length
over time.  (With collect=True, used by the tests, every tick is synchronous
and timed on the host.)
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
RING = 8  # ticks the host may run ahead of the GPU


@dataclasses.dataclass
class Episode:
    id: int
    capacity: int
    n_steps: int
    msgs_per_step: int
    arrival: float             # seconds (wall clock) or tick index (virtual clock)
    base: int = -1             # first message of the episode in the payload buffer
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


def footprint_bytes(capacity: int, trade_capacity: int) -> int:
    """Resident HBM an admitted episode holds: book state, trade log, counters."""
    k = 1
    while 32 * k < capacity:
        k *= 2
    return 48 * 32 * k + 32 * trade_capacity + 8 * 24 + 64


class _Pool:
    """Resident slots of one capacity class (numpy bookkeeping, one stream)."""

    def __init__(self, capacity, slots, trade_capacity, depth, collect):
        self.capacity, self.slots, self.depth = capacity, slots, depth
        self.stream = torch.cuda.Stream()
        with torch.cuda.stream(self.stream):
            self.engine = Engine(slots, capacity, trade_capacity, stream=self.stream)
            # one packed upload per tick: [start | count | ids (int32 pairs)]
            self.d_pack = torch.empty(3 * slots, dtype=torch.int64, device="cuda")
            self.d_start = self.d_pack[:slots]
            self.d_cnt = self.d_pack[slots:2 * slots]
            self.d_ids = self.d_pack[2 * slots:].view(torch.int32)
            self.levels = [torch.empty((slots, depth), dtype=torch.int32, device="cuda")
                           for _ in range(4)]
            self.d_tcount = torch.empty(slots, dtype=torch.int64, device="cuda")
            self.d_slot = torch.arange(slots, dtype=torch.int32, device="cuda")
        # a ring of pinned staging sets, so the host can run ahead of the GPU;
        # a set is reused only after the event recorded behind its copies
        self.ring = []
        for _ in range(RING):
            pack = torch.empty(3 * slots, dtype=torch.int64).pin_memory()
            self.ring.append(dict(pack=pack, np=pack.numpy(), used=torch.cuda.Event(),
                                  t0=torch.cuda.Event(enable_timing=True),
                                  t1=torch.cuda.Event(enable_timing=True), busy=False))
        self.ring_pos = 0
        self.lat = []  # (GPU ms of a timed tick, episodes in it)
        self.free = list(range(slots - 1, -1, -1))
        self.ep = np.full(slots, -1, np.int64)      # episode index in the slot, -1 free
        self.step = np.zeros(slots, np.int64)
        self.n_steps = np.zeros(slots, np.int64)
        self.mps = np.zeros(slots, np.int64)
        self.base = np.zeros(slots, np.int64)
        self.n_active = 0
        self.collect = collect

    def _retire_slot(self, st):
        """Wait for a staging set's tick to finish and record its GPU time."""
        st["used"].synchronize()
        if st.get("timed"):
            st["t1"].synchronize()
            self.lat.append((st["t0"].elapsed_time(st["t1"]), st["n"]))
        st["busy"] = False
        st["timed"] = False

    def flush(self):
        for st in self.ring:
            if st["busy"]:
                self._retire_slot(st)

    def admit(self, idx: int, ep: Episode):
        s = self.free.pop()
        self.ep[s], self.step[s] = idx, 0
        self.n_steps[s], self.mps[s], self.base[s] = ep.n_steps, ep.msgs_per_step, ep.base
        self.n_active += 1
        with torch.cuda.stream(self.stream):
            self.engine.reset_books(self.d_slot[s:s + 1])

    def launch_step(self, d_msgs, timing=False):
        """One step of every active slot, asynchronously on this pool's stream.
        Returns (active slots, messages, (start, end) events or None)."""
        act = np.flatnonzero(self.ep >= 0).astype(np.int32)
        n = len(act)
        cnt = self.mps[act]
        st = self.ring[self.ring_pos]
        self.ring_pos = (self.ring_pos + 1) % len(self.ring)
        if st["busy"]:
            self._retire_slot(st)
        sl = self.slots
        buf = st["np"]
        buf[:n] = self.base[act] + self.step[act] * cnt
        buf[sl:sl + n] = cnt
        buf[2 * sl:].view(np.int32)[:n] = act
        s = ctypes.c_void_p(self.stream.cuda_stream)
        p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
        ev = None
        with torch.cuda.stream(self.stream):
            st["timed"] = timing
            st["n"] = n
            if timing:
                ev = (st["t0"], st["t1"])
                ev[0].record(self.stream)
            self.d_pack.copy_(st["pack"], non_blocking=True)
            st["used"].record(self.stream)
            st["busy"] = True
            rc = lib().lob_process_segments(self.engine.h, p(d_msgs), p(self.d_start),
                                            p(self.d_cnt), p(self.d_ids), n, s)
            if rc != 0:
                raise RuntimeError("lob_process_segments failed")
            lob_get_levels(self.engine.h, self.depth, *self.levels, stream=self.stream)
            if self.collect:
                lib().lob_get_trades(self.engine.h, None, p(self.d_tcount), s)
            if timing:
                ev[1].record(self.stream)
        return act, int(cnt.sum()), ev


class Server:
    """Continuous batching over per-capacity slot pools with HBM admission."""

    def __init__(self, capacities=(100, 250, 500), hbm_budget=2 << 30, trade_capacity=2048,
                 depth=10, seed=20230829, max_slots=4096, collect=False):
        import lobgen
        self.lobgen = lobgen
        self.params = lobgen.make_params(seed, "pm1")
        self.depth = depth
        self.budget = hbm_budget
        self.fp = {c: footprint_bytes(c, trade_capacity) for c in capacities}
        self.pools = {c: _Pool(c, min(max_slots, max(1, hbm_budget // self.fp[c])),
                               trade_capacity, depth, collect)
                      for c in capacities}
        self.used = 0
        self.collect = collect
        self.records = collections.defaultdict(list)  # episode id -> per-step outputs
        self.final_books = {}

    def load(self, episodes):
        """Accept requests: generate every episode's message windows (stream id =
        episode id) into one HBM payload buffer.  Returns its size in bytes."""
        counts = np.array([e.n_steps * e.msgs_per_step for e in episodes], np.int64)
        gen = self.lobgen.DeviceStreams(self.params, len(episodes),
                                        stream_ids=[e.id for e in episodes])
        self.d_msgs, off = gen.advance(counts)
        off = off.cpu().numpy()
        for e, b in zip(episodes, off[:-1]):
            e.base = int(b)
        torch.cuda.synchronize()
        return int(counts.sum()) * MSG_BYTES

    def _can_admit(self, ep):
        pool = self.pools.get(ep.capacity)
        if pool is None:
            raise ValueError("no pool for capacity %d" % ep.capacity)
        return bool(pool.free) and self.used + self.fp[ep.capacity] <= self.budget

    def run(self, episodes, clock="wall", max_ticks=None):
        """Serve `episodes` (arrival in seconds for clock='wall', in ticks for
        clock='virtual'); returns a report dict."""
        payload = self.load(episodes)
        order = sorted(range(len(episodes)), key=lambda i: episodes[i].arrival)
        pending = collections.deque(order)
        waiting = []
        lat, weights, queue_len = [], [], []
        steps_done = msgs_done = 0
        max_active = max_used = 0
        tick = 0
        t0 = time.perf_counter()
        while pending or waiting or any(p.n_active for p in self.pools.values()):
            now = (time.perf_counter() - t0) if clock == "wall" else float(tick)
            while pending and episodes[pending[0]].arrival <= now:
                waiting.append(pending.popleft())
            still = []
            for i in waiting:  # first fit, in arrival order
                ep = episodes[i]
                if self._can_admit(ep):
                    self.pools[ep.capacity].admit(i, ep)
                    self.used += self.fp[ep.capacity]
                    ep.admitted = now
                else:
                    still.append(i)
            waiting = still
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
                launched = [(p, *p.launch_step(self.d_msgs)) for p in busy]
                for p in busy:
                    p.stream.synchronize()
                te = time.perf_counter()
                lat.append(te - ts)
                weights.append(active)
            else:
                # the host runs ahead; each pool's tick is timed on the GPU
                te = time.perf_counter()
                launched = [(p, *p.launch_step(self.d_msgs, timing=True)) for p in busy]
            steps_done += active
            msgs_done += sum(m for _, _, m, _ in launched)
            if self.collect:
                self._record(episodes, launched)
            now_after = (te - t0) if clock == "wall" else float(tick)
            for p, act, _, _ in launched:
                p.step[act] += 1
                for s in act[p.step[act] >= p.n_steps[act]]:
                    ep = episodes[int(p.ep[s])]
                    if self.collect:
                        self._final_book(p, int(s), ep)
                    ep.done = now_after
                    p.ep[s] = -1
                    p.n_active -= 1
                    p.free.append(int(s))
                    self.used -= self.fp[ep.capacity]
            tick += 1
            if max_ticks is not None and tick >= max_ticks:
                break
        torch.cuda.synchronize()
        for p in self.pools.values():
            p.flush()
            for ms, n in p.lat:
                lat.append(ms / 1e3)
                weights.append(n)
            p.lat = []
        wall = time.perf_counter() - t0
        lat_ms = np.repeat(np.asarray(lat) * 1e3, weights) if lat else np.zeros(1)
        waits = [e.admitted - e.arrival for e in episodes if not math.isnan(e.admitted)]
        return {"episodes": len(episodes), "episode_steps": steps_done, "messages": msgs_done,
                "payload_bytes": payload, "wall_s": wall, "ticks": tick,
                "steps_per_s": steps_done / wall, "msgs_per_s": msgs_done / wall,
                "p50_step_ms": float(np.percentile(lat_ms, 50)),
                "p99_step_ms": float(np.percentile(lat_ms, 99)),
                "mean_batch": float(np.mean(weights)) if weights else 0.0,
                "admission_wait_p50": float(np.percentile(waits, 50)) if waits else 0.0,
                "admission_wait_p99": float(np.percentile(waits, 99)) if waits else 0.0,
                "max_queue": max(q for _, q in queue_len) if queue_len else 0,
                "max_active": max_active, "max_hbm_bytes_admitted": max_used,
                "queue": queue_len}

    def _record(self, episodes, launched):
        for p, act, _, _ in launched:
            lv = [x.cpu().numpy() for x in p.levels]
            tc = p.d_tcount.cpu().numpy()
            for s in act:
                ep = episodes[int(p.ep[s])]
                self.records[ep.id].append((tuple(x[s].tolist() for x in lv), int(tc[s])))

    def _final_book(self, p, s, ep):
        bk = p.engine.book()
        p.stream.synchronize()
        self.final_books[ep.id] = {k: v[s].cpu().numpy().copy() for k, v in bk.items()}
