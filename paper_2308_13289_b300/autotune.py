"""Launch-shape autotuner for the batched processing kernel.

Sweeps warps per CTA (books in flight per CTA) and the staged chunk size
(messages per bulk copy) on a short prefix of the caller's own workload, and
caches the fastest shape per (device, capacity, number of books, mean messages
per book) in a JSON file.  Every shape computes the same result; only the
time differs.
"""
from __future__ import annotations

import json
import os

import torch

from . import Engine, LobError

CACHE_ENV = "LOB_AUTOTUNE_CACHE"
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_autotune_cache.json")

# non-powers of two too: with large books, shared memory decides how many
# warps fit on an SM, and all books resident at once (one wave) is what counts
WARPS = (1, 2, 3, 4, 6, 7, 8, 16)
CHUNKS = (32, 64, 128, 256)


def cache_path() -> str:
    return os.environ.get(CACHE_ENV, DEFAULT_CACHE)


def cache_key(device_name: str, capacity: int, n_books: int, mean_msgs: float) -> str:
    # book counts and stream lengths bucketed to powers of two
    nb = 1 << max(0, int(n_books - 1).bit_length())
    mm = 1 << max(0, int(max(1, mean_msgs) - 1).bit_length())
    return "%s|cap%d|books%d|msgs%d" % (device_name, capacity, nb, mm)


def load_cache(path=None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path=None) -> None:
    path = path or cache_path()
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(n_books, capacity, msgs, offsets, book_ids=None, trade_capacity=None, reps=3,
         warps=WARPS, chunks=CHUNKS, use_cache=True, mean_msgs=None):
    """Time every valid (warps, chunk) on `msgs`/`offsets` (device tensors, a
    prefix of the real workload) and return {'warps', 'chunk', 'ms', 'table'}."""
    dev = torch.cuda.get_device_name()
    if mean_msgs is None:
        mean_msgs = float((offsets[-1] - offsets[0]).item()) / max(1, offsets.numel() - 1)
    key = cache_key(dev, capacity, n_books, mean_msgs)
    if use_cache:
        hit = load_cache().get(key)
        if hit:
            return dict(hit, cached=True, key=key)
    if trade_capacity is None:
        seg = float((offsets[-1] - offsets[0]).item()) / max(1, offsets.numel() - 1)
        trade_capacity = int(seg) + 64
    e = Engine(n_books, capacity, trade_capacity)
    table = []
    for w in warps:
        for c in chunks:
            try:
                e.set_launch(w, c, 0)
            except LobError:
                continue
            times = []
            for r in range(reps + 1):
                e.reset()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                e.process_batch(msgs, offsets, book_ids)
                b.record()
                torch.cuda.synchronize()
                if r:
                    times.append(a.elapsed_time(b))
            table.append({"warps": w, "chunk": c, "ms": min(times)})
    e.close()
    if not table:
        raise RuntimeError("no launch shape fits this device")
    best = min(table, key=lambda t: t["ms"])
    res = {"warps": best["warps"], "chunk": best["chunk"], "ms": best["ms"], "table": table}
    if use_cache:
        cache = load_cache()
        cache[key] = res
        save_cache(cache)
    return dict(res, cached=False, key=key)


def apply(engine: Engine, shape: dict) -> None:
    engine.set_launch(shape["warps"], shape["chunk"], 0)
