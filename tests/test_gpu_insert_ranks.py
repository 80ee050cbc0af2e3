"""A limit order resting at every priority rank of a side, for every book
layout.

Each book holds one side of `f` resting orders (priority order = OID order),
then receives one more limit order on that side whose price puts it before
or after each price level in turn, or behind the whole side; a market order
from the other side then takes the first three orders and part of the
fourth.  The levels are either single orders (so every rank is a level
boundary) or runs of one to three equal prices (so the new order also lands
behind equal-priced orders, Sec. 4.2's time priority).  The fills include the
boundaries of a lane's slots and of the shared-memory book's 64-order window
(31 to 34, 62 to 66, 127 to 129) and full sides, where the full-side rule
evicts the worst order or rejects the new one.

CPU: the oracle puts the new order at every rank 0..f of a side that is not
full, and a full side evicts exactly when the new price is strictly better
than the worst one.  GPU: the CUDA path against the oracle, bit-exact, at
capacities on both sides of each slot-count boundary, under both rules.
"""
import functools

import numpy as np
import pytest

import lobgen
import oracle
from engine_harness import assert_same, run_both

BID, ASK = 1, -1
CAPS = [1, 2, 7, 32, 33, 64, 100, 128, 129, 256, 257, 500, 512]
SPECIAL = (1, 2, 31, 32, 33, 34, 62, 63, 64, 65, 66, 127, 128, 129)


def fills_for(cap):
    return sorted({f for f in SPECIAL + (0, cap - 2, cap - 1, cap) if 0 <= f <= cap})


def level_sizes(f, mixed, rng):
    sizes = []
    while sum(sizes) < f:
        sizes.append(int(rng.integers(1, 4)) if mixed else 1)
    if sizes:
        sizes[-1] -= sum(sizes) - f
    return [s for s in sizes if s > 0]


@functools.lru_cache(maxsize=2)
def rank_books(cap, seed=11, sweep=True):
    """Messages and offsets of every (side, fill, arrangement, target) book,
    plus per book (side, f, new price, the rank its price gives it; a full
    side keeps the new order only when that rank is below the capacity)."""
    rng = np.random.default_rng(seed + cap)
    rows, off, meta = [], [0], []
    for side in (BID, ASK):
        better = 1 if side == BID else -1  # a better price is higher for bids
        for f in fills_for(cap):
            for mixed in (False, True):
                sizes = level_sizes(f, mixed, rng)
                prices = [10_000 - better * 2 * i for i in range(len(sizes))]
                starts = np.concatenate([[0], np.cumsum(sizes)]).astype(int)
                targets = []  # (new price, rank it takes)
                for i, p in enumerate(prices):
                    targets.append((p + better, int(starts[i])))     # before level i
                    targets.append((p, int(starts[i + 1])))          # behind level i
                worst = prices[-1] if prices else 10_000
                targets.append((worst - better * (1 if prices else 0), f))  # behind the side
                for P, rank in targets:
                    t = 1_000
                    oid = 1
                    for i, p in enumerate(prices):
                        for _ in range(sizes[i]):
                            rows.append((1, side, p, 10 + oid, oid, oid % 7, t))
                            oid += 1
                            t += 10
                    rows.append((1, side, P, 500, 9_999, 3, t))
                    t += 10
                    if sweep:
                        take = sum(10 + k for k in range(1, 4)) + 1
                        rows.append((4, -side, 0, take, 8_888, 4, t))
                    off.append(len(rows))
                    meta.append((side, f, P, rank))
    msgs = np.array(rows, dtype=lobgen.MSG_DTYPE)
    return msgs, np.array(off, dtype=np.int64), meta


def test_new_order_takes_every_rank_in_the_oracle():
    for cap in (7, 33, 100, 129):
        msgs, off, meta = rank_books(cap, sweep=False)
        o = oracle.Oracle(len(meta), cap, 8, 0)
        o.process(msgs, off)
        bk = o.book()
        seen = {}
        for b, (side, f, P, rank) in enumerate(meta):
            s = 0 if side == BID else 1
            n = int(bk["count"][b, s])
            oids = list(bk["oid"][b, s, :n])
            if f < cap:
                assert n == f + 1 and oids.index(9_999) == rank, (cap, b)
                seen.setdefault((side, f), set()).add(rank)
            elif rank < cap:  # strictly better than the worst order: evicts it
                assert n == cap and oids.index(9_999) == rank and f not in oids, (cap, b)
            else:  # not better than the worst: rejected
                assert n == cap and 9_999 not in oids, (cap, b)
        for (side, f), ranks in seen.items():
            assert ranks == set(range(f + 1)), (cap, side, f)


@pytest.mark.gpu
@pytest.mark.parametrize("rule", [0, 1])
@pytest.mark.parametrize("cap", CAPS)
def test_insert_ranks_match_oracle(cap, rule):
    msgs, off, meta = rank_books(cap)
    g, r = run_both(msgs, off, cap, 8, rule)
    assert_same(g, r)
    c = dict(zip(oracle.COUNTERS, r["counters"].sum(0)))
    assert c["rested"] >= len(meta)  # every book rests its side, most the new order too
    if rule == 0:
        assert c["evicted"] > 0
    assert c["rejected"] > 0
