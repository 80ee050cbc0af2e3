"""Shared-memory ("grouped") books under pressure: sides filled to capacity
(the full-side rule evicting or rejecting on most adds), inserts far below
the top (the add's count and order move cross several 64-order windows),
cancels at every depth, and market orders that sweep across groups of 128.

The streams are hand-built with numpy (not the order-flow generator): limit
prices spread over a wide band so that adds land at every priority rank;
OIDs are unique and cancels name earlier ids on their own side (some already
gone, so some cancels miss).  CPU: the oracle shows that each case really
stresses what it is meant to.  GPU: the CUDA path against the oracle,
bit-exact, at capacities on both sides of the slot-count boundaries
(129 and 256 hold 256 slots, 257 to 512 hold 512).
"""
import numpy as np
import pytest

import lobgen
import oracle
from engine_harness import assert_same, run_both

BID, ASK = 1, -1
CAPS = [129, 256, 257, 400, 512]


def pressure_streams(n_books, n_msgs, seed):
    """Per book: 70 % limit adds (one in ten marketable), 27 % cancels or
    deletes of earlier ids, 3 % market orders large enough to take several
    orders at once.  Adds outpace removals, so the sides fill up."""
    rng = np.random.default_rng(seed)
    out = np.zeros(n_books * n_msgs, dtype=lobgen.MSG_DTYPE)
    k = 0
    for _ in range(n_books):
        ids = {BID: [], ASK: []}
        qty = {}
        oid, t = 1, 0
        for _ in range(n_msgs):
            t += 1 + int(rng.integers(0, 1000))
            u = rng.random()
            side = BID if rng.random() < 0.5 else ASK
            if u < 0.70:
                if rng.random() < 0.1:  # marketable: crosses into the other side
                    px = int(rng.integers(10_000, 10_060)) if side == BID else \
                        int(rng.integers(9_941, 10_001))
                else:  # resting anywhere in a wide band
                    px = int(rng.integers(9_000, 10_000)) if side == BID else \
                        int(rng.integers(10_001, 11_001))
                q = int(rng.integers(1, 200))
                out[k] = (1, side, px, q, oid, int(rng.integers(1, 50)), t)
                ids[side].append(oid)
                qty[oid] = q
                oid += 1
            elif u < 0.97 and ids[side]:
                target = ids[side][int(rng.integers(0, len(ids[side])))]
                full = rng.random() < 0.4
                q = qty[target] if full else int(rng.integers(1, qty[target] + 1))
                out[k] = (3 if full else 2, side, 0, q, target, 0, t)
            else:
                q = int(rng.integers(200, 1_500))
                out[k] = (4, side, 0, q, oid, int(rng.integers(1, 50)), t)
                oid += 1
            k += 1
    off = np.arange(0, n_books * n_msgs + 1, n_msgs, dtype=np.int64)
    return out, off


@pytest.mark.parametrize("rule", [0, 1])
def test_pressure_streams_stress_full_sides_and_sweeps(rule):
    msgs, off = pressure_streams(4, 6000, 5)
    o = oracle.Oracle(4, 257, 20_000, rule)
    o.process(msgs, off)
    c = dict(zip(oracle.COUNTERS, o.counters().sum(0)))
    if rule == 0:
        assert c["evicted"] > 1000
    else:
        assert c["rejected"] > 1000
    assert c["cancel_hit"] > 500 and c["cancel_miss"] > 100
    # market orders take several orders each on average
    assert c["trades"] > 2 * c["market"]
    assert (o.book()["count"] == 257).any()


@pytest.mark.gpu
@pytest.mark.parametrize("rule", [0, 1])
@pytest.mark.parametrize("cap", CAPS)
def test_gpu_grouped_books_under_pressure(cap, rule):
    msgs, off = pressure_streams(12, 6000, 100 + cap + rule)
    g, r = run_both(msgs, off, cap, 20_000, rule, depth=16)
    assert_same(g, r)
