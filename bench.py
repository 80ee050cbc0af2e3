"""Benchmark of the batched order-book engine on one B300 (or N, one rank each).

Default workload: replay_1024x100k -- 1,024 independent books of capacity 100,
10^5 synthetic messages per book (the config the headline metric is quoted on).
One step = the whole hot path over the batch: all books from empty through all
their messages (add / cancel / delete / market matching, trade log written),
then the top-10 levels of every book.

Forms timed on the same data:
  persistent  one launch per step: a persistent grid pulls books from a device
              work queue and keeps each book in shared memory for its whole
              stream (the reported `value`);
  plain       one launch per 100-message chunk (1,000 launches per step), book
              state to and from HBM each launch;
  plain_graph the plain form's 1,000 launches replayed from a CUDA graph.

`--impl reference` times the CPU oracle (the test-suite's checker, plain C++)
on the host cores on a bounded sample of the same workload.

Under torchrun every rank runs its own 1,024 books (weak scaling, no
collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("messages/sec (1 B300, bit-exact) batched-persistent vs plain; env steps/sec; "
          "p50/p99 step ms")
UNIT = "msgs/s"
DATA = "synthetic: seeded counter-based order-flow generator standing in for LOBSTER replay data"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="engine", choices=["engine", "reference"])
    ap.add_argument("--workload", default="replay_1024x100k")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-form legs")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--oracle-books", type=int, default=1024,
                    help="books of the CPU-baseline sample and of the full-size parity check "
                         "(full streams; the default takes every book of the headline workload)")
    ap.add_argument("--launch", default="", help="warps,chunk,ctas_per_sm override")
    ap.add_argument("--capacity", type=int, default=0,
                    help="book capacity override for the replay workloads (1..512)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the uneven / RL-environment / serving workloads")
    ap.add_argument("--serving-window", type=float, default=2.0,
                    help="seconds of Poisson arrivals in the serving workload")
    ap.add_argument("--serving-budget-mib", type=int, default=32,
                    help="HBM budget of the serving leg in which admission binds")
    ap.add_argument("--rl-forms", default="all",
                    help="RL workload legs to run: all, or a comma list of per_step, "
                         "persistent, graph, policy (a profiler can then select one)")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers

def dist_env():
    from paper_2308_13289_b300 import dist as ldist
    return ldist.rank_world()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", "lob_clocks_%d_%d.csv" % (os.getpid(), index))

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


COUNTER_RECORD = os.path.join("profiles", "k_process_replay_1024x100k_counters.txt")


def measured_counters():
    """ncu counters of one headline k_process launch from the committed
    record: DRAM bytes (read + write) and warp-instructions executed, with the
    messages of that launch.  None once the kernel sources have changed since
    the counters were taken (the record holds their hash)."""
    import hashlib
    path = os.path.join(ROOT, COUNTER_RECORD)
    try:
        kv = dict(line.split(":", 1) for line in open(path)
                  if ":" in line and not line.startswith("#"))
        h = hashlib.sha256()
        for src in kv["sources"].split():
            with open(os.path.join(ROOT, src), "rb") as f:
                h.update(f.read())
        if h.hexdigest() != kv["sources_sha256"].strip():
            return None
        return {"dram_bytes": int(kv["dram_bytes_read"]) + int(kv["dram_bytes_write"]),
                "inst_executed": int(kv["smsp_inst_executed"]),
                "messages": int(kv["messages"])}
    except (OSError, KeyError, ValueError):
        return None


def issue_roofline(inst_per_msg, msgs_per_s, sm_mhz, source, sms=None):
    """Fraction of the GPU's instruction-issue capacity a kernel uses: warp-
    instructions per message x messages per second, over (SMs x 4 schedulers,
    one warp-instruction per cycle each, x the median SM clock sampled during
    the timed region)."""
    if sms is None:
        import torch
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    if inst_per_msg is None or not sm_mhz:
        return {"bound": "issue", "inst_per_msg": inst_per_msg, "frac": None, "source": source}
    achieved = inst_per_msg * msgs_per_s
    peak = sms * 4 * sm_mhz * 1e6
    return {"bound": "issue", "inst_per_msg": round(inst_per_msg, 2),
            "achieved": round(achieved / 1e9, 2), "peak": round(peak / 1e9, 2),
            "unit": "G warp-instructions/s", "frac": round(achieved / peak, 4),
            "sms": sms, "sm_mhz": sm_mhz, "source": source}


def workload_streams(name, rank):
    import lobgen
    w = lobgen.WORKLOADS[name]
    n = w["n_books"]
    if w.get("msgs"):
        counts = np.full(n, w["msgs"], np.int64)
    else:
        counts = lobgen.lognormal_counts(n, w["seed"])
    params = lobgen.make_params(w["seed"], w["mid_walk"])
    from paper_2308_13289_b300 import dist as ldist
    sid = ldist.stream_ids(rank, n)
    msgs, off = lobgen.generate(params, counts, stream_ids=sid)
    return w, params, counts, msgs, off, sid


def trade_capacity_for(counts):
    # enough for every trade of the longest stream (fills/message < 0.7 here)
    return int(min(1 << 20, max(1024, int(counts.max() * 0.75) + 1024)))


# ------------------------------------------------------------------ engine arm

def run_engine(args):
    import torch

    import paper_2308_13289_b300 as eng
    from paper_2308_13289_b300 import build as eng_build

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    eng_build.build()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    w, params, counts, msgs, off, sid = workload_streams(args.workload, rank)
    n = len(counts)
    total_msgs = int(off[-1])
    cap = args.capacity or w["capacity"]
    tcap = trade_capacity_for(counts)
    depth = 10

    d_msgs = eng.messages_to_device(msgs)
    d_off = torch.from_numpy(off).cuda()
    stream = torch.cuda.current_stream()

    # ---------------- persistent form
    e = eng.Engine(n, cap, tcap)
    launch = None
    if args.launch:
        e.set_launch(*[int(x) for x in args.launch.split(",")])
        launch = {"override": args.launch}
    elif counts.min() == counts.max() and counts[0] >= 5000:
        # autotune warps/CTA and chunk on the first 5,000 messages of every book
        from paper_2308_13289_b300 import autotune
        per = int(counts[0])
        pre = d_msgs.view(n, per, 8)[:, :5000].contiguous().view(-1, 8)
        pre_off = torch.arange(0, n * 5000 + 1, 5000, dtype=torch.int64, device="cuda")
        shape = autotune.tune(n, cap, pre, pre_off, trade_capacity=5000, mean_msgs=per)
        autotune.apply(e, shape)
        launch = {"warps_per_cta": shape["warps"], "chunk_msgs": shape["chunk"],
                  "autotuned_on": "first 5,000 messages of every book", "cached": shape["cached"],
                  "table_ms": {"%d,%d" % (t["warps"], t["chunk"]): round(t["ms"], 3)
                               for t in shape["table"]}}
        del pre, pre_off
    lv_out = [torch.empty((n, depth), dtype=torch.int32, device="cuda") for _ in range(4)]

    def step_persistent(ev=None):
        e.reset()
        if ev is not None:
            ev[0].record(stream)
        e.process_batch(d_msgs, d_off)
        if ev is not None:
            ev[1].record(stream)
        eng.lob_get_levels(e.h, depth, *lv_out)

    for _ in range(args.warmup):
        step_persistent()
    torch.cuda.synchronize()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = e.launch_count()
    torch.cuda.synchronize()
    barrier()
    with nvtx("persistent"):
        t0.record(stream)
        for i in range(args.steps):
            step_persistent(kev[i])
        t1.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = e.launch_count() - launches0
    ms_total = t0.elapsed_time(t1)
    kernel_ms = float(np.mean([a.elapsed_time(b) for a, b in kev]))
    ms_total = max_over_ranks(ms_total, world)
    ms_step = ms_total / args.steps

    # outputs of the last step for the parity check and the roofline bytes
    ctr, st = e.stats()
    trades_per_step = int(ctr[:, 6].sum().item())
    status = int(st.item())

    # ---------------- plain form: one launch per 100-message chunk
    plain = plain_graph = None
    chunk = w.get("chunk", 100)
    uniform = bool((counts == counts[0]).all()) and counts[0] % chunk == 0
    if not args.no_plain and uniform:
        per = int(counts[0])
        nch = per // chunk
        cm = torch.empty_like(d_msgs)
        cm.view(nch, n, chunk, 8).copy_(d_msgs.view(n, nch, chunk, 8).transpose(0, 1))
        seg = torch.arange(0, n * chunk + 1, chunk, dtype=torch.int64, device="cuda")
        ep = eng.Engine(n, cap, tcap, append_trades=True)
        base = cm.data_ptr()
        rowbytes = n * chunk * 32

        def step_plain():
            ep.reset()
            for c in range(nch):
                rc = eng.lib().lob_process_batch(
                    ep.h, ctypes.c_void_p(base + c * rowbytes), ctypes.c_void_p(seg.data_ptr()),
                    None, n, ctypes.c_void_p(stream.cuda_stream))
                if rc != 0:
                    raise eng.LobError(rc, "lob_process_batch")
            eng.lob_get_levels(ep.h, depth, *lv_out)

        plain = time_steps(step_plain, args, stream, barrier, world, name="plain")
        plain["launches_per_step"] = nch + 1
        # same result as the persistent form
        plain["bit_exact_vs_persistent"] = same_results(e, ep, depth)
        # graph-captured plain form
        g = torch.cuda.CUDAGraph()
        s2 = torch.cuda.Stream()
        s2.wait_stream(stream)
        with torch.cuda.stream(s2):
            step_plain()  # warm the capture stream
            torch.cuda.synchronize()
            with torch.cuda.graph(g, stream=s2):
                ep.reset()
                for c in range(nch):
                    rc = eng.lib().lob_process_batch(
                        ep.h, ctypes.c_void_p(base + c * rowbytes),
                        ctypes.c_void_p(seg.data_ptr()), None, n,
                        ctypes.c_void_p(s2.cuda_stream))
                    if rc != 0:
                        raise eng.LobError(rc, "lob_process_batch")
                eng.lob_get_levels(ep.h, depth, *lv_out, stream=s2)
        stream.wait_stream(s2)
        plain_graph = time_steps(lambda: g.replay(), args, stream, barrier, world,
                                 name="plain_graph")
        plain_graph["launches_per_step"] = nch + 1
        plain_graph["bit_exact_vs_persistent"] = same_results(e, ep, depth)
        del g
        ep.close()
        del cm
    clk = clocks.stop()

    # ---------------- end to end through host buffers (pinned), copies timed
    e2e = None
    if not args.no_e2e:
        h_msgs = torch.from_numpy(np.ascontiguousarray(msgs).view(np.int32).reshape(-1, 8)).pin_memory()
        h_off = torch.from_numpy(off).pin_memory()
        h_lv = [torch.empty((n, depth), dtype=torch.int32).pin_memory() for _ in range(4)]
        h_cnt = torch.empty(n, dtype=torch.int64).pin_memory()
        d_cnt = torch.empty(n, dtype=torch.int64, device="cuda")

        per_book = int(counts[0]) if counts.min() == counts.max() else 0
        e2e_chunk = 2000
        before = snapshot_results(e, depth)  # the persistent form's last step

        def step_e2e():
            e.reset()
            if per_book:
                # message chunks copied from pinned host memory while the
                # previous chunk is processed (lob_process_host)
                e.process_host(h_msgs, per_book, e2e_chunk)
            else:
                d_msgs.copy_(h_msgs, non_blocking=True)
                d_off.copy_(h_off, non_blocking=True)
                e.process_batch(d_msgs, d_off)
            eng.lob_get_levels(e.h, depth, *lv_out)
            eng.lob_get_trades(e.h, None, d_cnt)
            for h, d in zip(h_lv, lv_out):
                h.copy_(d, non_blocking=True)
            h_cnt.copy_(d_cnt, non_blocking=True)

        r = time_steps(step_e2e, args, stream, barrier, world, steps=max(3, args.steps // 2),
                       name="e2e")
        e2e = {"value": total_msgs * world / (r["ms_per_step"] / 1e3), "unit": UNIT,
               "ms_per_step": r["ms_per_step"],
               "h2d_bytes_per_step": int(h_msgs.numel() * 4 + (0 if per_book else h_off.numel() * 8)),
               "d2h_bytes_per_step": int(4 * n * depth * 4 + n * 8),
               "path": ("lob_process_host: %d-message chunks copied while the previous chunk "
                        "is processed" % e2e_chunk) if per_book else
                       "copy of all messages, then lob_process_batch",
               "bit_exact_vs_persistent": all(
                   torch.equal(x, y) for x, y in zip(before, snapshot_results(e, depth)))}

    overflow = overflow_stats(e)

    # ---------------- parity on a sample of books + CPU baseline (rank 0 only)
    cpu = parity = None
    if rank == 0 and args.oracle_books > 0:
        cpu, parity = cpu_baseline_and_parity(e, msgs, off, counts, cap, tcap, depth,
                                              args.oracle_books, w)
        if world > 1:  # the CPU baseline is reported at N = 1 only; parity at every N
            cpu = None

    # ---------------- roofline of the processing kernel
    peak, peak_kind = measured_peaks()
    state_bytes = 2 * n * eng_book_bytes(cap)
    alg_bytes = 32 * total_msgs + 32 * trades_per_step + state_bytes + 8 * (n + 1)
    achieved = alg_bytes / (kernel_ms / 1e3) / 1e9
    counters = (measured_counters() if args.workload == "replay_1024x100k" and cap == 100
                else None)
    roof = {"bound": "hbm", "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 5),
            "traffic": counters["dram_bytes"] if counters else None,
            "kernel": "k_process<%d>" % (eng_book_bytes(cap) // (48 * 32)),
            "kernel_ms": round(kernel_ms, 4), "algorithmic_bytes_per_launch": int(alg_bytes),
            "peak_kind": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)"}
    # the roofline that binds this kernel: instruction issue of each book's
    # serial chain (warp-instructions per message from the committed ncu record)
    ipm = counters["inst_executed"] / counters["messages"] if counters else None
    roof["issue"] = issue_roofline(ipm, total_msgs / (kernel_ms / 1e3), clk.get("sm_mhz"),
                                   COUNTER_RECORD + " (smsp__inst_executed.sum)" if counters
                                   else "no counter record for these kernel sources")

    extras = None
    # the other workloads are single-GPU legs: a run on N > 1 GPUs measures the
    # headline's scaling only and holds the GPUs no longer than that needs
    if not args.no_extras and args.workload == "replay_1024x100k" and world == 1:
        e.close()
        del d_msgs
        torch.cuda.empty_cache()
        extras = {}
        for key, fn in (("replay_book_sweep", lambda a, r: run_sweep(a, r, ipm, clk)),
                        ("uneven_4096_lognormal", run_uneven), ("rl_exec_8192x400", run_rl),
                        ("serving_mix", run_serving), ("ablation_paper_literal", run_ablation)):
            with nvtx(key):
                extras[key] = fn(args, rank)
        e = eng.Engine(1, cap, 1)

    if rank == 0:
        value = total_msgs * world / (ms_step / 1e3)
        line = {"metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "int32", "data": DATA,
                "config": {"workload": args.workload, "n_books_per_gpu": n,
                           "capacity": cap, "messages_per_step_per_gpu": total_msgs,
                           "trades_per_step_per_gpu": trades_per_step,
                           "trade_capacity": tcap, "form": "persistent", "launch": launch,
                           "l2": "inputs larger than L2 (%.2f GB of messages)" % (total_msgs * 32 / 1e9),
                           "seed": w["seed"],
                           # independent books: every rank runs its own, no data-path collective
                           "parallelism": "book-sharded x%d" % world},
                "plain": plain, "plain_graph": plain_graph,
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": int(launches), "clocks": clk, "parity": parity,
                "overflow": overflow, "device_status": status, "workloads": extras}
        print(json.dumps(line))
    e.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def replay_oracle_check(e, params, ids, counts, cap, tcap, depth=10, chunk=4096, logs=4):
    """Every book of a replay run against the oracle replaying the same seeded
    streams (host copies, all host threads), `chunk` books at a time: the
    canonical books, top `depth` levels, counters and trade counts of every
    book, and the whole trade logs of the first `logs` books of each chunk.
    Returns (verdict, oracle seconds)."""
    import torch

    import lobgen
    import oracle
    n = len(counts)
    bk = {k: v.cpu().numpy() for k, v in e.book().items()}
    lv = [x.cpu().numpy() for x in e.levels(depth)]
    ctr = e.stats()[0].cpu().numpy()
    gt, gc = e.trades()
    tc = gc.cpu().numpy()
    ok, secs = True, 0.0
    for c0 in range(0, n, chunk):
        sel = np.arange(c0, min(n, c0 + chunk))
        hm, hoff = lobgen.generate(params, counts[sel], stream_ids=ids[sel])
        o = oracle.Oracle(len(sel), cap, tcap)
        t = time.perf_counter()
        o.process(hm, hoff)
        secs += time.perf_counter() - t
        for k, v in o.book().items():
            ok &= np.array_equal(bk[k][sel], v)
        for g, x in zip(lv, o.levels(depth)):
            ok &= np.array_equal(g[sel], x)
        ok &= np.array_equal(ctr[sel], o.counters())
        ot, oc = o.trades()
        ok &= np.array_equal(tc[sel], oc)
        m = min(logs, len(sel))
        ok &= np.array_equal(gt[c0:c0 + m].cpu().numpy(),
                             ot[:m].view(np.int32).reshape(m, tcap, 8))
        del o, hm, hoff, ot
        if not ok:
            break
    del gt
    torch.cuda.empty_cache()
    return bool(ok), secs


def run_sweep(args, rank, inst_per_msg=None, clk=None, sizes=(1024, 4096, 16384), per=10_000):
    """The replay workload's generator at 10^4 messages per book and a growing
    number of books (persistent form, autotuned shape): where the kernel
    leaves the regime in which each book's serial chain sets the time, and
    how the HBM and issue fractions move."""
    import torch

    import lobgen
    import paper_2308_13289_b300 as eng
    from paper_2308_13289_b300 import autotune
    w = lobgen.WORKLOADS["replay_1024x10k"]
    cap = w["capacity"]
    params = lobgen.make_params(w["seed"], w["mid_walk"])
    peak, peak_kind = measured_peaks()
    res = {"messages_per_book": per, "capacity": cap, "seed": w["seed"],
           "peak_hbm_gbs": peak, "inst_per_msg_source": "headline ncu record"}
    for n in sizes:
        ids = np.arange(rank * n, (rank + 1) * n, dtype=np.uint64)
        gen = lobgen.DeviceStreams(params, n, stream_ids=ids)
        dm, doff = gen.advance([per] * n)
        del gen
        tcap = per // 2 + 1024
        e = eng.Engine(n, cap, tcap)
        pre_n = 2000
        pre = dm.view(n, per, 8)[:, :pre_n].contiguous().view(-1, 8)
        pre_off = torch.arange(0, n * pre_n + 1, pre_n, dtype=torch.int64, device="cuda")
        shape = autotune.tune(n, cap, pre, pre_off, trade_capacity=pre_n, mean_msgs=per)
        autotune.apply(e, shape)
        del pre, pre_off
        times = []
        for i in range(args.warmup + args.steps):
            e.reset()
            a, b = _events()
            a.record()
            e.process_batch(dm, doff)
            b.record()
            torch.cuda.synchronize()
            if i >= args.warmup:
                times.append(a.elapsed_time(b))
        ms = float(np.mean(times))
        ctr, st = e.stats()
        trades = int(ctr[:, 6].sum().item())
        total = n * per
        alg = 32 * total + 32 * trades + 2 * n * eng_book_bytes(cap) + 8 * (n + 1)
        rate = total / ms * 1e3
        row = {"n_books": n, "ms_per_step": round(ms, 4), "msgs_per_s": round(rate, 1),
               "launch": {"warps_per_cta": shape["warps"], "chunk_msgs": shape["chunk"]},
               "hbm_frac": round(alg / (ms / 1e3) / 1e9 / peak, 5),
               "issue": issue_roofline(inst_per_msg, rate, (clk or {}).get("sm_mhz"),
                                       "headline record's instructions per message"),
               "device_status": int(st.item())}
        if rank == 0:
            ok, secs = replay_oracle_check(e, params, ids, np.full(n, per, np.int64), cap, tcap)
            row["parity"] = {"books_checked": n, "bit_exact": ok, "oracle_s": round(secs, 2)}
        res["n%d" % n] = row
        e.close()
        del dm, doff
        torch.cuda.empty_cache()
    return res


def run_ablation(args, rank, name="replay_1024x10k"):
    """The design ablation on 1,024 books x 10^4 messages: this library's
    sorted warp sides (one persistent launch) against the paper's own
    formulation on the GPU -- unsorted arrays with full scans, branching on
    the message type, and with every branch run on a copy of the book (what
    vmap does) -- all bit-exact with one another."""
    import torch

    import lobgen
    import paper_2308_13289_b300 as eng
    w = lobgen.WORKLOADS[name]
    n, per, cap = w["n_books"], w["msgs"], w["capacity"]
    params = lobgen.make_params(w["seed"], w["mid_walk"])
    ids = np.arange(rank * n, (rank + 1) * n, dtype=np.uint64)
    gen = lobgen.DeviceStreams(params, n, stream_ids=ids)
    dm, doff = gen.advance([per] * n)
    del gen
    tcap = per
    total = n * per

    def timed(fn, reps):
        times = []
        for i in range(1 + reps):
            a, b = _events()
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            if i >= 1:
                times.append(a.elapsed_time(b))
        return float(np.mean(times))

    e = eng.Engine(n, cap, tcap)

    def sorted_form():
        e.reset()
        e.process_batch(dm, doff)

    res = {"workload": name, "n_books": n, "messages": total, "capacity": cap}
    ms = timed(sorted_form, max(3, args.steps))
    res["sorted_warp_sides"] = {"ms_per_step": round(ms, 4), "msgs_per_s": round(total / ms * 1e3, 1)}
    ref = {k: v.clone() for k, v in e.book().items()}
    _, ref_cnt = e.trades()
    e.close()
    for form, allb in (("literal_branching", False), ("literal_all_branches", True)):
        out = {}

        def lit():
            out["r"] = eng.literal_process(dm, doff, cap, tcap, eng.OVERFLOW_EVICT, allb)

        ms_l = timed(lit, 2)
        bk, _, cnt = out["r"]
        same = all(torch.equal(bk[k], ref[k]) for k in ref) and torch.equal(cnt, ref_cnt)
        res[form] = {"ms_per_step": round(ms_l, 4), "msgs_per_s": round(total / ms_l * 1e3, 1),
                     "slowdown_vs_sorted": round(ms_l / ms, 2), "bit_exact_vs_sorted": bool(same)}
        del out
    del dm, doff
    torch.cuda.empty_cache()
    return res


def run_uneven(args, rank):
    """4,096 books with lognormal message counts in ONE persistent launch whose
    work queue hands out books in natural order or longest first."""
    import torch

    import lobgen
    import paper_2308_13289_b300 as eng
    w = lobgen.WORKLOADS["uneven_4096_lognormal"]
    n = w["n_books"]
    counts = lobgen.lognormal_counts(n, w["seed"])
    params = lobgen.make_params(w["seed"], w["mid_walk"])
    ids = np.arange(rank * n, (rank + 1) * n, dtype=np.uint64)
    tcap = trade_capacity_for(counts)
    import hashlib
    res = {"n_books": n, "messages": int(counts.sum()), "count_min": int(counts.min()),
           "count_max": int(counts.max()), "count_mean": float(counts.mean()),
           "counts_sha256": hashlib.sha256(counts.astype("<i8").tobytes()).hexdigest(),
           "seed": w["seed"]}
    for order in ("natural", "longest_first"):
        perm = np.arange(n) if order == "natural" else np.argsort(-counts, kind="stable")
        gen = lobgen.DeviceStreams(params, n, stream_ids=ids)
        dm, doff = gen.advance(counts[perm], ids=perm.astype(np.int32))
        d_ids = torch.from_numpy(perm.astype(np.int32)).cuda()
        e = eng.Engine(n, w["capacity"], tcap)
        if "launch" not in res:
            # autotune books per CTA and chunk size on every book's first 1,000
            # messages (every book has at least that many)
            from paper_2308_13289_b300 import autotune
            pre_n = 1000
            idx = (doff[:-1].unsqueeze(1) + torch.arange(pre_n, device="cuda")).reshape(-1)
            pre = dm.view(-1, 8)[idx].contiguous()
            pre_off = torch.arange(0, n * pre_n + 1, pre_n, dtype=torch.int64, device="cuda")
            shape = autotune.tune(n, w["capacity"], pre, pre_off, trade_capacity=pre_n,
                                  mean_msgs=float(counts.mean()))
            res["launch"] = {"warps_per_cta": shape["warps"], "chunk_msgs": shape["chunk"],
                             "autotuned_on": "first 1,000 messages of every book",
                             "cached": shape.get("cached", False)}
            del pre, idx
        autotune_shape = res["launch"]
        e.set_launch(autotune_shape["warps_per_cta"], autotune_shape["chunk_msgs"], 0)
        times = []
        for i in range(args.warmup + args.steps):
            e.reset()
            a, b = _events()
            a.record()
            e.process_batch(dm, doff, d_ids)
            b.record()
            torch.cuda.synchronize()
            if i >= args.warmup:
                times.append(a.elapsed_time(b))
        ms = float(np.mean(times))
        trades = int(e.stats()[0][:, 6].sum().item())
        # messages, trades, book state in and out, offsets and book ids
        alg = 32 * res["messages"] + 32 * trades + 2 * n * eng_book_bytes(w["capacity"]) + \
            8 * (n + 1) + 4 * n
        peak, _ = measured_peaks()
        res[order] = {"ms_per_step": round(ms, 4), "msgs_per_s": round(res["messages"] / ms * 1e3, 1),
                      "algorithmic_bytes": alg, "hbm_frac": round(alg / (ms / 1e3) / 1e9 / peak, 5)}
        if order == "longest_first" and rank == 0:
            # every book against the oracle replaying its own stream
            ok, secs = replay_oracle_check(e, params, ids, counts, w["capacity"], tcap)
            _, st = e.stats()
            res["parity"] = {"books_checked": n, "bit_exact": ok, "oracle_s": round(secs, 2),
                             "device_status": int(st.item())}
            res["overflow"] = overflow_stats(e)
        e.close()
        del dm, doff, gen
    return res


def env_oracle_check(w, params, ids, got, draws=None, actions=None, final=None, obs=None,
                     chunk=1024):
    """The oracle's environments (oracle.EnvOracle, all host threads) replay
    the episode of every environment, `chunk` environments at a time, from the
    host copy of the same seeded streams; every step's reward (by its bits),
    fills and four level arrays are compared with `got` (host arrays
    [steps, n, ...]); so are, when given, the final books and agent state
    (`final`) and, for the policy form (`actions`), the last step's
    observation (`obs`).  Returns the verdict (and the observation's)."""
    import lobgen
    import oracle
    steps, n = got["reward"].shape
    per = w["msgs_per_step"]
    ok, ok_obs = True, True
    for c0 in range(0, n, chunk):
        sel = np.arange(c0, min(n, c0 + chunk))
        hm, _ = lobgen.generate(params, [steps * per] * len(sel), stream_ids=ids[sel])
        rows = hm.reshape(len(sel), steps, per)
        offs = np.arange(0, len(sel) * per + 1, per)
        oenv = oracle.EnvOracle(len(sel), w["capacity"], 4096, n_steps=steps)
        tr = None
        for t in range(steps):
            stp = np.ascontiguousarray(rows[:, t, :]).reshape(-1)
            if actions is None:
                r_, lv, f_ = oenv.step(stp, offs, draws[t, sel], t)
            else:
                r_, lv, f_, tr = oenv.step(stp, offs, None, t, l1=True, actions=actions[t, sel])
            ok &= got["reward"][t, sel].tobytes() == r_.tobytes()
            ok &= np.array_equal(got["fills"][t, sel], f_)
            for k, x in zip(("bid_px", "bid_qty", "ask_px", "ask_qty"), lv):
                ok &= np.array_equal(got[k][t, sel], x)
        if final is not None:
            ost, op0 = oenv.state()
            ok &= np.array_equal(final["state"][sel], ost)
            ok &= final["p_init"][sel].tobytes() == op0.tobytes()
            for k, v in oenv.books.book().items():
                ok &= np.array_equal(final["books"][k][sel], v)
        if obs is not None:
            t_init = rows[:, 0, 0]["time_ns"].astype(np.int64)
            ok_obs &= oenv.observe(tr, per, t_init).tobytes() == obs[sel].tobytes()
        del oenv, hm, rows
        if not ok:
            break
    return (ok, ok_obs) if obs is not None else ok


def run_rl(args, rank, name="rl_exec_8192x400"):
    """8,192 execution environments x 400 steps x 100 data messages: one launch
    per step, the same 400 launches replayed from a CUDA graph, and one
    persistent launch for the whole episode."""
    import torch

    import lobgen
    import oracle
    import paper_2308_13289_b300 as eng
    w = lobgen.WORKLOADS[name]
    n, steps, per = w["n_books"], w["steps"], w["msgs_per_step"]
    params = lobgen.make_params(w["seed"], w["mid_walk"])
    ids = np.arange(rank * n, (rank + 1) * n, dtype=np.uint64)
    gen = lobgen.DeviceStreams(params, n, stream_ids=ids)
    dm, _ = gen.advance([steps * per] * n)
    del gen
    draws = lobgen.agent_draws_device(w["seed"] + 1, n, steps)
    e = eng.Engine(n, w["capacity"], 4096)
    env = eng.Env(e, n_steps=steps, msgs_per_step=per)
    out = env.outputs(steps)
    stride = steps * per

    def per_step():
        e.reset()
        env.reset()
        for t in range(steps):
            env.run(dm, stride, t, 1, draws[t:t + 1], out, row0=t)

    def persistent():
        e.reset()
        env.reset()
        env.run(dm, stride, 0, steps, draws, out)

    def snapshot():
        torch.cuda.synchronize()
        st, p0 = env.state()
        return [v.clone() for v in out.values()] + [st, p0] + list(e.book().values())

    res = {"n_envs": n, "steps": steps, "msgs_per_step": per, "seed": w["seed"]}
    want = set(args.rl_forms.split(",")) if args.rl_forms != "all" else {
        "per_step", "persistent", "graph", "policy"}
    ref = None
    forms = {}
    for name, form, fn in (("per_step_launches", "per_step", per_step),
                           ("persistent_episode", "persistent", persistent)):
        if form not in want:
            continue
        times = []
        for i in range(max(1, args.warmup) + max(2, args.steps // 3)):
            a, b = _events()
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            if i >= max(1, args.warmup):
                times.append(a.elapsed_time(b))
        forms[name] = float(np.mean(times))
        snap = snapshot()
        if ref is None:
            ref = snap
        else:
            res["persistent_equals_per_step"] = all(torch.equal(x, y) for x, y in zip(ref, snap))
    ran = {"per_step": "per_step_launches", "persistent": "persistent_episode"}
    missing = [f for f, leg in ran.items() if f in want and leg not in forms]
    if missing:
        raise RuntimeError("RL legs requested but not run: %s" % missing)
    if "persistent" in want:
        res["segments_per_episode"] = env.segments()
    if want != {"per_step", "persistent", "graph", "policy"}:
        # a subset of the legs (profiling): timings only
        for name, ms in forms.items():
            res[name] = {"ms_per_episode": round(ms, 3),
                         "env_steps_per_s": round(n * steps / ms * 1e3, 1)}
        env.close()
        e.close()
        del dm, out
        torch.cuda.empty_cache()
        return res
    # CUDA graph of the per-step form
    s2 = torch.cuda.Stream()
    s2.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s2):
        with torch.cuda.graph(g, stream=s2):
            per_step()
    torch.cuda.current_stream().wait_stream(s2)
    times = []
    for i in range(max(1, args.warmup) + max(2, args.steps // 3)):
        a, b = _events()
        a.record()
        g.replay()
        b.record()
        torch.cuda.synchronize()
        if i >= max(1, args.warmup):
            times.append(a.elapsed_time(b))
    forms["graph_per_step"] = float(np.mean(times))
    res["graph_equals_per_step"] = all(torch.equal(x, y) for x, y in zip(ref, snapshot()))
    del g
    std_out = {k: v.cpu().numpy() for k, v in out.items()}  # the stand-in agent's episode
    std_trades = int(e.stats()[0][:, 6].sum().item())
    st_, p0_ = env.state()
    std_final = dict(state=st_.cpu().numpy(), p_init=p0_.cpu().numpy(),
                     books={k: v.cpu().numpy() for k, v in e.book().items()})
    res["overflow"] = overflow_stats(e)
    # policy loop (Sec. 5.2.2-5.2.3): every step acts on four sizes and ends
    # with the step's level-1 trace and the observation vector, as a policy in
    # the loop needs; the sizes are seeded stand-ins for a policy's output
    gen_a = torch.Generator(device="cuda")
    gen_a.manual_seed(w["seed"] + 2)
    act = torch.rand((steps, n, 4), generator=gen_a, device="cuda") * 4.0
    l1 = torch.empty((1, n, per, 4), dtype=torch.int32, device="cuda")
    obs = torch.empty((n, 6 * per + 8), dtype=torch.float32, device="cuda")

    def policy_steps():
        e.reset()
        env.reset()
        for t in range(steps):
            env.run(dm, stride, t, 1, None, out, row0=t, l1=l1, actions=act[t:t + 1])
            env.observe(dm, stride, l1[0], obs)

    s3 = torch.cuda.Stream()
    s3.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s3):
        with torch.cuda.graph(g, stream=s3):
            policy_steps()
    torch.cuda.current_stream().wait_stream(s3)
    for name, fn in (("policy_per_step", policy_steps), ("policy_graph", g.replay)):
        times = []
        for i in range(max(1, args.warmup) + max(2, args.steps // 3)):
            a, b = _events()
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            if i >= max(1, args.warmup):
                times.append(a.elapsed_time(b))
        forms[name] = float(np.mean(times))
    del g
    policy_trades = int(e.stats()[0][:, 6].sum().item())
    # algorithmic bytes of an episode (what each form must move): the data
    # messages, the trades, the per-step outputs (levels, reward, fills), the
    # agent's input (draws; or actions, then the trace and the observation,
    # the trace read back by it), and the books' state in and out once per
    # launch
    depth = env.depth
    state = 2 * n * eng_book_bytes(w["capacity"])
    std_alg = n * steps * (per * 32 + 4 * depth * 4 + 4 + 16 + 4) + 32 * std_trades
    pol_alg = n * steps * (per * 32 + 4 * depth * 4 + 4 + 16 + 16 + 2 * 16 * per +
                           (6 * per + 8) * 4) + 32 * policy_trades + steps * state
    peak, _ = measured_peaks()
    for name, ms in forms.items():
        alg = pol_alg if name.startswith("policy") else \
            std_alg + (state if name == "persistent_episode" else steps * state)
        res[name] = {"ms_per_episode": round(ms, 3),
                     "env_steps_per_s": round(n * steps / ms * 1e3, 1),
                     "data_msgs_per_s": round(n * steps * per / ms * 1e3, 1),
                     "launches": (1 if name == "persistent_episode" else
                                  2 * steps if name.startswith("policy") else steps),
                     "algorithmic_bytes": alg,
                     "hbm_frac": round(alg / (ms / 1e3) / 1e9 / peak, 5)}
    if rank == 0:
        # every environment, every step, against the oracle's environments
        hd = lobgen.agent_draws(w["seed"] + 1, n, steps)
        t0 = time.time()
        ok = env_oracle_check(w, params, ids, std_out, draws=hd, final=std_final)
        res["parity"] = {"envs_checked": n, "steps_checked": steps, "bit_exact": bool(ok),
                         "compared": "every step's reward bits, fills and four level arrays; "
                                     "final books and agent state",
                         "oracle_s": round(time.time() - t0, 1)}
        t0 = time.time()
        ok, ok_obs = env_oracle_check(w, params, ids, {k: v.cpu().numpy() for k, v in out.items()},
                                      actions=act.cpu().numpy(), obs=obs.cpu().numpy())
        res["policy_parity"] = {"envs_checked": n, "steps_checked": steps, "bit_exact": bool(ok),
                                "final_observation_bit_exact": bool(ok_obs),
                                "oracle_s": round(time.time() - t0, 1)}
    env.close()
    e.close()
    del dm, out
    torch.cuda.empty_cache()
    return res


def run_serving(args, rank):
    """Poisson arrivals (2,000 episodes/s) of episodes with capacity 100/250/500,
    200..2,000 steps and 100..500 messages per step, served by continuous
    batching with admission by HBM footprint (book, trade log, counters,
    generator state and step window).  Two legs on the same requests: a 2 GiB
    budget that never binds, and a small budget under which admission decides
    (episodes queue, the queue length is sampled over time)."""
    import copy

    import torch

    import lobgen
    from paper_2308_13289_b300.serve import Server, sample_episodes
    w = lobgen.WORKLOADS["serving_mix"]
    eps = sample_episodes(w["rate"], args.serving_window, w["seed"] + rank, w["capacities"],
                          w["steps"], w["msgs_per_step"])
    res = {"episodes": len(eps), "window_s": args.serving_window, "seed": w["seed"] + rank,
           "offered_msgs_per_s": round(sum(e.n_steps * e.msgs_per_step for e in eps)
                                       / args.serving_window, 1),
           "offered_episode_steps_per_s": round(sum(e.n_steps for e in eps)
                                                / args.serving_window, 1)}
    # a sample checked against the oracle at full size: the shortest episode
    # of each capacity and the longest one (whole episodes are replayed on one
    # host thread)
    size = lambda e: e.n_steps * e.msgs_per_step  # noqa: E731
    sample = []
    for c in w["capacities"]:
        mine = [e for e in eps if e.capacity == c]
        if mine:
            sample.append(min(mine, key=size))
    if eps:
        sample.append(max(eps, key=size))
    # the third leg splits every capacity class at 300 messages per step: a
    # pool's tick lasts as long as its longest window, so short windows get
    # their own pools (latency against throughput: more pools, more host work
    # per tick)
    for leg, budget, buckets in (("uncontended", 2 << 30, ()),
                                 ("contended", args.serving_budget_mib << 20, ()),
                                 ("bucketed", 2 << 30, (300,))):
        srv = Server(capacities=w["capacities"], seed=w["seed"], hbm_budget=budget,
                     msgs_per_step=w["msgs_per_step"], capture_ids=[e.id for e in sample],
                     window_buckets=buckets)
        rep = srv.run([copy.copy(e) for e in eps], clock="wall")
        if rank == 0:
            rep["parity"] = serving_parity(srv, sample, w["seed"])
        q = rep.pop("queue")
        rep["queue_samples"] = [(round(t, 3), n) for t, n in q[::max(1, len(q) // 20)]]
        for k in ("wall_s", "steps_per_s", "msgs_per_s", "p50_step_ms", "p99_step_ms",
                  "p50_window_gen_ms", "admission_wait_p50", "admission_wait_p99"):
            if rep.get(k) is not None:
                rep[k] = round(rep[k], 4)
        for v in rep.get("per_capacity", {}).values():
            for k in ("p50_step_ms", "p99_step_ms"):
                v[k] = round(v[k], 4)
        res[leg] = rep
        del srv
        torch.cuda.empty_cache()
    return res


def serving_parity(srv, sample, seed, tcap=2048):
    """Final book and counters of each sampled episode against the oracle
    replaying the episode's stream (stream id = episode id) step by step."""
    import lobgen
    import oracle
    params = lobgen.make_params(seed, "pm1")
    ok, msgs = True, 0
    for ep in sample:
        hs = lobgen.HostStreams(params, 1, stream_ids=[ep.id])
        o = oracle.Oracle(1, ep.capacity, tcap)
        for _ in range(ep.n_steps):
            m, off = hs.advance([ep.msgs_per_step], threads=1)
            o.process(m, off, threads=1)
            msgs += len(m)
        got = srv.final_books.get(ep.id)
        if got is None:
            ok = False
            continue
        ok &= all(np.array_equal(v[0], got[k]) for k, v in o.book().items())
        ok &= np.array_equal(o.counters()[0], srv.final_counters[ep.id])
    return {"episodes_checked": len(sample), "messages": msgs, "bit_exact": bool(ok),
            "capacities": [e.capacity for e in sample]}


def eng_book_bytes(cap):
    k = 1
    while 32 * k < cap:
        k *= 2
    return 48 * 32 * k


def max_over_ranks(x, world):
    from paper_2308_13289_b300 import dist as ldist
    return x if world == 1 else ldist.max_over_ranks(x, device="cuda")


def nvtx(name):
    """NVTX range around a bench leg (lets a profiler select it by name)."""
    import contextlib

    import torch

    @contextlib.contextmanager
    def rng():
        torch.cuda.nvtx.range_push(name)
        try:
            yield
        finally:
            torch.cuda.nvtx.range_pop()
    return rng()


def time_steps(fn, args, stream, barrier, world, steps=None, name="leg"):
    import torch
    steps = steps or args.steps
    with nvtx(name):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms = max_over_ranks(a.elapsed_time(b), world) / steps
    return {"ms_per_step": round(ms, 4)}


def overflow_stats(e):
    """Fraction of messages that met the full-side rule (Sec. 4 overflow
    reading: rejected or evicting), from the engine's own counters."""
    import paper_2308_13289_b300 as eng
    ctr = e.stats()[0].sum(dim=0).cpu().numpy()
    c = dict(zip(eng.COUNTERS, (int(x) for x in ctr)))
    hits = c["rejected"] + c["evicted"]
    return {"full_side_rule_fraction": round(hits / max(1, c["msgs"]), 5),
            "rejected": c["rejected"], "evicted": c["evicted"], "messages": c["msgs"]}


def snapshot_results(e, depth):
    """Copies of every output of an engine: books, trade logs and counts,
    levels, counters."""
    b = e.book()
    t, c = e.trades()
    return [v.clone() for v in b.values()] + [t.clone(), c.clone()] + \
        [x.clone() for x in e.levels(depth)] + [e.stats()[0].clone()]


def same_results(e1, e2, depth):
    import torch
    b1, b2 = e1.book(), e2.book()
    t1, c1 = e1.trades()
    t2, c2 = e2.trades()
    l1, l2 = e1.levels(depth), e2.levels(depth)
    s1, s2 = e1.stats()[0], e2.stats()[0]
    ok = all(torch.equal(b1[k], b2[k]) for k in b1) and torch.equal(c1, c2) and \
        torch.equal(t1, t2) and all(torch.equal(x, y) for x, y in zip(l1, l2)) and \
        torch.equal(s1, s2)
    return bool(ok)


def cpu_baseline_and_parity(e, msgs, off, counts, cap, tcap, depth, n_sample, w):
    """Time the CPU oracle (as it stands) on the first `n_sample` books' full
    streams with all host threads, and compare the GPU's results for those
    books element by element."""
    import oracle
    n_sample = min(n_sample, len(counts))
    threads = oracle.default_threads()
    sub_off = off[:n_sample + 1]
    sub = msgs[:int(sub_off[-1])]
    o = oracle.Oracle(n_sample, cap, tcap)
    t = time.perf_counter()
    o.process(sub, sub_off, threads=threads)
    dt = time.perf_counter() - t
    n_msgs = int(sub_off[-1])
    cpu = {"value": round(n_msgs / dt, 1), "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": oracle_sample_text(n_sample, counts, n_msgs), "seconds": round(dt, 3),
           "cpu_model": cpu_model(), "single_thread": oracle_single_thread(msgs, off, cap, tcap)}
    # parity
    bk = e.book()
    gl = e.levels(depth)
    ctr, _ = e.stats()
    ok = True
    ob = o.book()
    for k, v in ob.items():
        ok &= np.array_equal(bk[k][:n_sample].cpu().numpy(), v)
    for gv, ov in zip(gl, o.levels(depth)):
        ok &= np.array_equal(gv[:n_sample].cpu().numpy(), ov)
    ok &= np.array_equal(ctr[:n_sample].cpu().numpy(), o.counters())
    gt, gc = e.trades()
    ot, oc = o.trades()
    ok &= np.array_equal(gc[:n_sample].cpu().numpy(), oc)
    n_cmp = min(n_sample, 32)
    ok &= np.array_equal(gt[:n_cmp].cpu().numpy(),
                         ot[:n_cmp].view(np.int32).reshape(n_cmp, tcap, 8))
    parity = {"books_checked": n_sample, "trade_logs_checked": n_cmp, "bit_exact": bool(ok)}
    return cpu, parity


def oracle_sample_text(n_sample, counts, n_msgs):
    return ("first %d of %d books, full %s-message streams (%d messages), std::map oracle, "
            "one std::thread per host core" % (
                n_sample, len(counts), "{:,}".format(int(counts[0])) if (counts == counts[0]).all()
                else "lognormal", n_msgs))


def oracle_single_thread(msgs, off, cap, tcap, n1=16):
    """The oracle on one thread over the first n1 books' full streams (after
    one untimed run of the same books, so that the figure is not a cold start)."""
    import oracle
    n1 = min(n1, len(off) - 1)
    oracle.Oracle(n1, cap, tcap).process(msgs[:int(off[n1])], off[:n1 + 1], threads=1)
    o1 = oracle.Oracle(n1, cap, tcap)
    t = time.perf_counter()
    o1.process(msgs[:int(off[n1])], off[:n1 + 1], threads=1)
    dt1 = time.perf_counter() - t
    return {"value": round(int(off[n1]) / dt1, 1), "unit": UNIT,
            "sample": "first %d books, full streams (%d messages), 1 thread" % (n1, int(off[n1])),
            "seconds": round(dt1, 3)}


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


# ------------------------------------------------------------------ reference arm

def run_reference(args):
    """The CPU oracle, as it stands, on the host cores: each step processes the
    same bounded sample as the engine arm's cpu_baseline (the first
    --oracle-books books' full streams, all host threads), and the
    single-thread figure is measured the same way too."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    w, params, counts, msgs, off, sid = workload_streams(args.workload, 0)
    n_sample = min(max(1, args.oracle_books), len(counts))
    sub_off = off[:n_sample + 1]
    sub = msgs[:int(sub_off[-1])]
    cap, tcap = args.capacity or w["capacity"], trade_capacity_for(counts)
    threads = oracle.default_threads()
    n_msgs = int(sub_off[-1])

    def step():
        o = oracle.Oracle(n_sample, cap, tcap)
        o.process(sub, sub_off, threads=threads)
        o.levels(10)

    for _ in range(args.warmup):
        step()
    t = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t) / args.steps
    value = n_msgs / dt
    cpu = {"value": round(value, 1), "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": oracle_sample_text(n_sample, counts, n_msgs) + " per step",
           "cpu_model": cpu_model(),
           "single_thread": oracle_single_thread(msgs, off, cap, tcap)}
    line = {"metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": DATA, "impl": "reference",
            "config": {"workload": args.workload, "n_books_per_gpu": len(counts),
                       "capacity": cap, "form": "cpu oracle sample"},
            "cpu_baseline": cpu,
            "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_single(args):
    """One non-headline workload on its own, printed as its own JSON line."""
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    from paper_2308_13289_b300 import build as eng_build
    eng_build.build()
    wl = args.workload
    if wl.startswith("rl_exec"):
        r = run_rl(args, rank, wl)
        leg = r.get("persistent_episode") or r.get("per_step_launches") or {}
        value, unit = leg.get("env_steps_per_s"), "env-steps/s"
    elif wl.startswith("uneven"):
        r = run_uneven(args, rank)
        value, unit = r["natural"]["msgs_per_s"], UNIT
    elif wl == "ablation":
        r = run_ablation(args, rank)
        value, unit = r["sorted_warp_sides"]["msgs_per_s"], UNIT
    else:
        r = run_serving(args, rank)
        value, unit = r["uncontended"]["steps_per_s"], "episode-steps/s"
    if rank == 0:
        print(json.dumps({"metric": METRIC, "value": value, "unit": unit, "n_gpus": world,
                          "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
                          "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": DATA,
                          "config": {"workload": wl}, "result": r}))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload.startswith(("rl_exec", "uneven", "serving", "ablation")):
        run_single(args)
    else:
        run_engine(args)


if __name__ == "__main__":
    main()
