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

Every tick advances ALL admitted episodes by one step.  Per capacity class:
one generator launch writes the active slots' windows on the pool's generator
stream, one lob_process_batch launch applies them and one
lob_get_levels_books launch reports the levels of the same slots (not of the
whole pool) on the pool's processing stream.  The windows are
double-buffered, so the generator produces tick k+1 while tick k is being
processed; the classes run on their own streams and overlap on the device.

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


def _p(t, byte_off=0):
    return ctypes.c_void_p(t.data_ptr() + byte_off)


_cudart = None


def _memcpy_h2d_async():
    """cudaMemcpyAsync of the CUDA runtime torch loaded (raw pointers and
    stream handle: a tick's upload without torch's stream bookkeeping)."""
    global _cudart
    if _cudart is None:
        lib = ctypes.CDLL("libcudart.so.%d" % int(torch.version.cuda.split(".")[0]))
        fn = lib.cudaMemcpyAsync
        fn.restype = ctypes.c_int
        fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int,
                       ctypes.c_void_p]
        _cudart = fn
    return _cudart


class _Pool:
    """Resident slots of one capacity class: an engine context over all slots,
    per-slot generator state, double-buffered step windows, two streams."""

    def __init__(self, capacity, slots, trade_capacity, depth, params, max_mps, collect):
        self.capacity, self.slots, self.depth, self.params = capacity, slots, depth, params
        self.max_mps = max_mps
        # processing ahead of window generation when both have blocks waiting
        # for an SM (the step latency is the processing's)
        self.stream = torch.cuda.Stream(priority=-1)  # processing
        self.gstream = torch.cuda.Stream(priority=0)  # window generation
        S = slots
        # packed per-tick upload (int64 words): offsets [S+1] | counts [S] |
        # restart stream ids [S] | active slot ids (int32) [S] | restart slots (int32) [S]
        self.o_cnt, self.o_sid, self.o_ids = S + 1, 2 * S + 1, 3 * S + 1
        self.o_rid = self.o_ids + (S + 1) // 2
        self.pack_words = self.o_rid + (S + 1) // 2
        with torch.cuda.stream(self.stream):
            self.engine = Engine(slots, capacity, trade_capacity, stream=self.stream)
            self.g_states = torch.zeros(S * lobgen.STATE_BYTES, dtype=torch.uint8, device="cuda")
            self.g_pools = torch.zeros(S * params.pool_cap * lobgen.POOL_ENTRY_BYTES,
                                       dtype=torch.uint8, device="cuda")
            self.geo_px = torch.from_numpy(lobgen.GEO_PX.view(np.int64)).cuda()
            self.geo_q = torch.from_numpy(lobgen.GEO_Q.view(np.int64)).cuda()
            self.win = [torch.empty((S * max_mps, 8), dtype=torch.int32, device="cuda")
                        for _ in range(2)]
            self.d_pack = [torch.empty(self.pack_words, dtype=torch.int64, device="cuda")
                           for _ in range(2)]
            self.levels = [torch.empty((S, depth), dtype=torch.int32, device="cuda")
                           for _ in range(4)]
            self.d_tcount = torch.empty(S, dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()
        self.reserved_bytes = (S * (book_bytes(capacity) + 8 + 32 * trade_capacity + 8
                                    + 8 * N_COUNTERS + GEN_STATE_BYTES)
                               + 2 * S * max_mps * MSG_BYTES)
        # device addresses and handles used every tick (the buffers never move)
        self.h_ps = ctypes.c_void_p(self.stream.cuda_stream)
        self.h_gs = ctypes.c_void_p(self.gstream.cuda_stream)
        self.a_win = [_p(w) for w in self.win]
        self.a_pack = [dict(off=_p(d), cnt=_p(d, 8 * self.o_cnt), sid=_p(d, 8 * self.o_sid),
                            ids=_p(d, 8 * self.o_ids), rid=_p(d, 8 * self.o_rid))
                       for d in self.d_pack]
        self.a_states, self.a_pools = _p(self.g_states), _p(self.g_pools)
        self.a_geo_px, self.a_geo_q = _p(self.geo_px), _p(self.geo_q)
        self.a_levels = [_p(x) for x in self.levels]
        self.a_tcount = _p(self.d_tcount)
        self.params_ref = ctypes.byref(self.params)
        self.memcpy = _memcpy_h2d_async()
        self.ev_gen = [torch.cuda.Event() for _ in range(2)]   # windows k ready
        self.ev_used = [torch.cuda.Event() for _ in range(2)]  # windows k consumed
        self.ring = []
        for _ in range(RING):
            pack = torch.empty(self.pack_words, dtype=torch.int64).pin_memory()
            self.ring.append(dict(pack=pack, np=pack.numpy(), a_pack=_p(pack),
                                  copied=torch.cuda.Event(),
                                  g0=torch.cuda.Event(enable_timing=True),
                                  g1=torch.cuda.Event(enable_timing=True),
                                  t0=torch.cuda.Event(enable_timing=True),
                                  t1=torch.cuda.Event(enable_timing=True),
                                  busy=False, timed=False, n=0))
        self.ring_pos = 0
        self.tick = 0
        self.lat = []      # (GPU ms of a timed tick's processing, episodes in it)
        self.gen_ms = []   # GPU ms of a timed tick's window generation
        self.free = list(range(slots - 1, -1, -1))
        self.ep = np.full(slots, -1, np.int64)      # episode index in the slot, -1 free
        self.step = np.zeros(slots, np.int64)
        self.n_steps = np.zeros(slots, np.int64)
        self.mps = np.zeros(slots, np.int64)
        self.restart = []  # (slot, stream id) admitted since the last tick
        self.n_active = 0
        self.collect = collect

    def _retire(self, st):
        """Wait until a staging set's upload has landed; record its timings."""
        st["copied"].synchronize()
        if st["timed"]:
            st["t1"].synchronize()
            self.lat.append((st["t0"].elapsed_time(st["t1"]), st["n"]))
            self.gen_ms.append(st["g0"].elapsed_time(st["g1"]))
        st["busy"] = st["timed"] = False

    def flush(self):
        for st in self.ring:
            if st["busy"]:
                self._retire(st)

    def admit(self, idx: int, ep: Episode):
        if ep.msgs_per_step > self.max_mps:
            raise ValueError("episode %d: %d messages per step above the pool's %d"
                             % (ep.id, ep.msgs_per_step, self.max_mps))
        s = self.free.pop()
        self.ep[s], self.step[s] = idx, 0
        self.n_steps[s], self.mps[s] = ep.n_steps, ep.msgs_per_step
        self.restart.append((s, ep.id))
        self.n_active += 1

    def launch_step(self, timing=False):
        """One step of every active slot, asynchronously: windows on the
        generator stream, processing and levels on the processing stream.
        Returns (active slots, messages)."""
        act = np.flatnonzero(self.ep >= 0).astype(np.int32)
        n = len(act)
        cnt = self.mps[act]
        st = self.ring[self.ring_pos]
        self.ring_pos = (self.ring_pos + 1) % len(self.ring)
        if st["busy"]:
            self._retire(st)
        buf = st["np"]
        buf[0] = 0
        np.cumsum(cnt, out=buf[1:n + 1])
        buf[self.o_cnt:self.o_cnt + n] = cnt
        nr = len(self.restart)
        if nr:
            rs = np.array(self.restart, dtype=np.int64)
            buf[self.o_sid:self.o_sid + nr] = rs[:, 1]
            buf[self.o_rid:].view(np.int32)[:nr] = rs[:, 0]
        buf[self.o_ids:].view(np.int32)[:n] = act
        self.restart = []
        k = self.tick & 1
        ap = self.a_pack[k]
        lg = lobgen.cuda_lib()
        lb = lib()
        gs, ps = self.gstream, self.stream
        # generator stream: the windows of this tick (buffer k is free once
        # the processing of tick-2 has consumed it)
        gs.wait_event(self.ev_used[k])
        if self.memcpy(ap["off"], st["a_pack"], 8 * self.pack_words, 1, self.h_gs) != 0:
            raise RuntimeError("cudaMemcpyAsync of the tick's upload failed")
        st["copied"].record(gs)
        st["busy"], st["timed"], st["n"] = True, timing, n
        if timing:
            st["g0"].record(gs)
        if nr and lg.lobgen_dev_init_ids(self.params_ref, nr, ap["rid"], ap["sid"], self.a_states,
                                         self.h_gs) != 0:
            raise RuntimeError("lobgen_dev_init_ids failed")
        if lg.lobgen_dev_advance(self.params_ref, self.a_geo_px, self.a_geo_q, n, ap["ids"],
                                 self.a_states, self.a_pools, ap["cnt"], ap["off"], self.a_win[k],
                                 self.h_gs) != 0:
            raise RuntimeError("lobgen_dev_advance failed")
        if timing:
            st["g1"].record(gs)
        self.ev_gen[k].record(gs)
        # processing stream
        ps.wait_event(self.ev_gen[k])
        if timing:
            st["t0"].record(ps)
        h = self.engine.h
        if nr and lb.lob_reset_books(h, ap["rid"], nr, self.h_ps) != 0:
            raise RuntimeError("lob_reset_books failed")
        if lb.lob_process_batch(h, self.a_win[k], ap["off"], ap["ids"], n, self.h_ps) != 0:
            raise RuntimeError("lob_process_batch failed")
        if lb.lob_get_levels_books(h, ap["ids"], n, self.depth, *self.a_levels, self.h_ps) != 0:
            raise RuntimeError("lob_get_levels_books failed")
        if self.collect:
            lb.lob_get_trades(h, None, self.a_tcount, self.h_ps)
        if timing:
            st["t1"].record(ps)
        self.ev_used[k].record(ps)
        self.tick += 1
        return act, int(cnt.sum())

    def capture_final(self):
        """The pool's books and counters as they stand once the work queued so
        far has run (device tensors, filled in stream order)."""
        with torch.cuda.stream(self.stream):
            bk = self.engine.book()
            ctr, _ = self.engine.stats()
        return bk, ctr


class Server:
    """Continuous batching over per-capacity slot pools with HBM admission."""

    def __init__(self, capacities=(100, 250, 500), hbm_budget=2 << 30, trade_capacity=2048,
                 depth=10, seed=20230829, max_slots=4096, collect=False, keep_final=False,
                 msgs_per_step=(100, 500), capture_ids=None):
        self.params = lobgen.make_params(seed, "pm1")
        self.depth = depth
        self.budget = hbm_budget
        self.tcap = trade_capacity
        self.collect = collect
        self.keep_final = keep_final or collect
        self.capture_ids = set(capture_ids) if capture_ids else set()
        lo, hi = msgs_per_step
        self.pools = {}
        for c in capacities:
            # as many slots as the budget holds of the smallest episodes
            slots = int(min(max_slots, max(1, hbm_budget // footprint_bytes(c, trade_capacity, lo))))
            self.pools[c] = _Pool(c, slots, trade_capacity, depth, self.params, hi, collect)
        self.used = 0
        self.records = collections.defaultdict(list)  # episode id -> per-step outputs
        self.final_books = {}
        self.final_counters = {}

    def footprint(self, ep):
        return footprint_bytes(ep.capacity, self.tcap, ep.msgs_per_step)

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
            pool = self.pools.get(ep.capacity)
            if pool is None:
                raise ValueError("no pool for capacity %d" % ep.capacity)
            if pool.free and self.used + fps[i] <= self.budget:
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
                launched = [(p, *p.launch_step(timing=True)) for p in busy]
            steps_done += active
            msgs_done += sum(m for _, _, m in launched)
            now_after = (te - t0) if clock == "wall" else float(tick)
            for p, act, _ in launched:
                p.step[act] += 1
                ended = act[p.step[act] >= p.n_steps[act]]
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
                    p.free.append(int(s))
                    self.used -= fps[i]
            tick += 1
            if max_ticks is not None and tick >= max_ticks:
                break
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        gen_ms = []
        per_pool = {}
        for c, p in self.pools.items():
            p.flush()
            if p.lat:
                pl = np.repeat(np.asarray([ms for ms, _ in p.lat]), [n for _, n in p.lat])
                per_pool[c] = {"p50_step_ms": float(np.percentile(pl, 50)),
                               "p99_step_ms": float(np.percentile(pl, 99)),
                               "episode_steps": int(len(pl))}
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
                "slots": {c: p.slots for c, p in self.pools.items()},
                "per_capacity": per_pool,
                "queue": queue_len}

    def _record(self, episodes, launched):
        for p, act, _ in launched:
            lv = [x.cpu().numpy() for x in p.levels]
            tc = p.d_tcount.cpu().numpy()
            for s in act:
                ep = episodes[int(p.ep[s])]
                self.records[ep.id].append((tuple(x[s].tolist() for x in lv), int(tc[s])))
