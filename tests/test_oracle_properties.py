"""Invariants and closed-form special cases of the CPU oracle (Sec. 4.1-4.2).

Checked after EVERY message of seeded streams:
  * the book is never crossed (best bid < best ask);
  * both sides are in priority order, FIFO (arrival) inside a level;
  * no side holds more than N orders, no OID is live twice;
  * quantity conservation: limit qty + market qty submitted
      = 2 * traded + cancelled + rejected + evicted + resting + market dropped;
  * every trade has a positive quantity at the standing order's own limit
    price, at a price the aggressor accepts, and fills within one level
    happen oldest first.
"""
import numpy as np
import pytest

import lobgen
import oracle
from golden_format import side_rows


def _check_book(bk, cap, b=0):
    bids, asks = side_rows(bk, b, 0), side_rows(bk, b, 1)
    assert len(bids) <= cap and len(asks) <= cap
    if bids and asks:
        assert bids[0][0] < asks[0][0], "crossed book"
    for rows, desc in ((bids, True), (asks, False)):
        for x, y in zip(rows, rows[1:]):
            if desc:
                assert x[0] >= y[0]
            else:
                assert x[0] <= y[0]
            if x[0] == y[0]:
                assert x[4] < y[4], "FIFO violated inside a level"
        oids = [r[2] for r in rows]
        assert len(oids) == len(set(oids))
        assert all(r[1] > 0 for r in rows)
    return bids, asks


def _conservation(c, resting):
    lhs = c["limit_qty"] + c["market_qty"]
    rhs = (2 * c["traded_qty"] + c["cancelled_qty"] + c["rejected_qty"] + c["evicted_qty"]
           + resting + c["market_discarded_qty"])
    assert lhs == rhs


@pytest.mark.parametrize("cap,walk,rule", [(100, "pm1", 0), (10, "three", 0), (6, "pm1", 1)])
def test_invariants_after_every_message(cap, walk, rule):
    p = lobgen.make_params(7000 + cap, walk)
    n_msgs = 2500
    msgs, _ = lobgen.generate(p, [n_msgs])
    limit_price = {}
    o = oracle.Oracle(1, cap, 4096, rule)
    one = np.array([0, 1], np.int64)
    for i in range(n_msgs):
        m = msgs[i:i + 1]
        if m["type"][0] == 1:
            limit_price[int(m["oid"][0])] = int(m["price"][0])
        o.process(m, one, threads=1)
        bk = o.book()
        _check_book(bk, cap)
        c = dict(zip(oracle.COUNTERS, o.counters()[0]))
        _conservation(c, int(o.resting_qty()[0]))
        tr, cnt = o.trades()
        n = int(cnt[0])
        if n:
            t = tr[0][:n]
            assert (t["qty"] > 0).all()
            assert (t["oid_aggr"] == m["oid"][0]).all()
            assert (t["time_ns"] == m["time_ns"][0]).all()
            for k in range(n):
                assert t["price"][k] == limit_price[int(t["oid_stand"][k])]
            if m["type"][0] == 1:
                if m["side"][0] == 1:
                    assert (t["price"] <= m["price"][0]).all()
                else:
                    assert (t["price"] >= m["price"][0]).all()
            # price monotone in execution order, oldest first inside a level
            px = t["price"].astype(np.int64)
            step = np.diff(px) * (1 if m["side"][0] == 1 else -1)
            assert (step >= 0).all()
            for k in range(1, n):
                if px[k] == px[k - 1]:
                    assert t["oid_stand"][k] > t["oid_stand"][k - 1]
            assert int(t["qty"].sum()) <= int(m["qty"][0])


def test_market_larger_than_side_trades_everything_in_priority_order():
    """Closed form: a market order at least as large as the whole opposite side
    empties it and trades every standing order once, in priority order, each for
    its full quantity (Sec. 4.2 item 3 with the Sec. 4.1 loop run to exhaustion)."""
    p = lobgen.make_params(4242, "pm1")
    msgs, off = lobgen.generate(p, [3000] * 4)
    o = oracle.Oracle(4, 100, 512)
    o.process(msgs, off)
    before = o.book()
    c_before = o.counters()
    mk = []
    for b in range(4):
        mk.append((4, 1, 0, 2_000_000_000, 900_000 + b, 5, 10 ** 15))
    mk = oracle.messages(mk)
    o.process(mk, np.arange(5, dtype=np.int64))
    after = o.book()
    tr, cnt = o.trades()
    for b in range(4):
        asks = side_rows(before, b, 1)
        assert int(cnt[b]) == len(asks)
        got = [(int(t["price"]), int(t["qty"]), int(t["oid_stand"])) for t in tr[b][:len(asks)]]
        assert got == [(a[0], a[1], a[2]) for a in asks]
        assert after["count"][b, 1] == 0
        assert side_rows(after, b, 0) == side_rows(before, b, 0)
        c = dict(zip(oracle.COUNTERS, o.counters()[b] - c_before[b]))
        assert c["market_discarded_qty"] == 2_000_000_000 - sum(a[1] for a in asks)


def test_adds_and_cancels_without_crossing_give_the_live_multiset():
    """Closed form: with no crossing and no overflow the book is exactly the
    set of added orders minus cancelled quantity, bids sorted by (-P, arrival),
    asks by (P, arrival)."""
    rng = np.random.default_rng(5)
    rows, live = [], {}
    t = 0
    for oid in range(1, 400):
        t += 1
        if live and rng.random() < 0.35:
            tgt = int(rng.choice(sorted(live)))
            s, p, q, tm = live[tgt]
            dq = int(rng.integers(1, 2 * q + 1))
            rows.append((2 if rng.random() < 0.5 else 3, s, p, dq, tgt, 1, t))
            if dq >= q:
                del live[tgt]
            else:
                live[tgt] = (s, p, q - dq, tm)
        else:
            s = 1 if rng.random() < 0.5 else -1
            p = int(rng.integers(90, 100)) if s == 1 else int(rng.integers(101, 111))
            q = int(rng.integers(1, 50))
            rows.append((1, s, p, q, oid, 7, t))
            live[oid] = (s, p, q, t)
    o = oracle.Oracle(1, 1000, 16)
    m = oracle.messages(rows)
    o.process(m, np.array([0, len(m)], np.int64))
    bk = o.book()
    exp_b = sorted([(p, q, oid, 7, tm) for oid, (s, p, q, tm) in live.items() if s == 1],
                   key=lambda r: (-r[0], r[4]))
    exp_a = sorted([(p, q, oid, 7, tm) for oid, (s, p, q, tm) in live.items() if s == -1],
                   key=lambda r: (r[0], r[4]))
    assert side_rows(bk, 0, 0) == exp_b
    assert side_rows(bk, 0, 1) == exp_a
    assert o.trades()[1][0] == 0


def test_rules_agree_when_capacity_never_binds():
    """With capacity above the number of adds, evict and reject rules give the
    same books and trades and never fire."""
    p = lobgen.make_params(99, "pm1")
    msgs, off = lobgen.generate(p, [1500] * 3)
    res = []
    for rule in (0, 1):
        o = oracle.Oracle(3, 2000, 4096, rule)
        o.process(msgs, off)
        res.append((o.book(), o.trades(), o.counters()))
    for k in res[0][0]:
        assert np.array_equal(res[0][0][k], res[1][0][k])
    assert np.array_equal(res[0][1][0], res[1][1][0])
    c = dict(zip(oracle.COUNTERS, res[0][2].sum(0)))
    assert c["evicted"] == 0 and c["rejected"] == 0


def test_chunked_calls_with_append_equal_one_call():
    """Splitting a stream into calls changes nothing when trades append."""
    p = lobgen.make_params(31337, "three")
    msgs, off = lobgen.generate(p, [2000] * 5)
    o1 = oracle.Oracle(5, 100, 4096)
    o1.process(msgs, off)
    o2 = oracle.Oracle(5, 100, 4096, append_trades=True)
    per = msgs.reshape(5, 2000)
    for c0 in range(0, 2000, 300):
        c1 = min(2000, c0 + 300)
        chunk = np.ascontiguousarray(per[:, c0:c1]).reshape(-1)
        o2.process(chunk, np.arange(0, 5 * (c1 - c0) + 1, c1 - c0, dtype=np.int64))
    for k, v in o1.book().items():
        assert np.array_equal(v, o2.book()[k])
    assert np.array_equal(o1.trades()[0], o2.trades()[0])
    assert np.array_equal(o1.counters(), o2.counters())


def test_set_book_roundtrip():
    p = lobgen.make_params(3, "pm1")
    msgs, off = lobgen.generate(p, [3000] * 2)
    o = oracle.Oracle(2, 100, 64)
    o.process(msgs, off)
    bk = o.book()
    o2 = oracle.Oracle(2, 100, 64)
    o2.set_book(bk)
    for k, v in o2.book().items():
        assert np.array_equal(v, bk[k])


def test_level1_trace_matches_levels_after_each_message():
    """The level-1 trace after message k equals level 0 of the top-level
    output computed on the book as it stands after message k."""
    p = lobgen.make_params(61, "pm1")
    msgs, _ = lobgen.generate(p, [600])
    o1 = oracle.Oracle(1, 20, 256)
    l1 = o1.process_l1(msgs, np.array([0, len(msgs)], np.int64))
    o2 = oracle.Oracle(1, 20, 256)
    one = np.array([0, 1], np.int64)
    for k in range(len(msgs)):
        o2.process(msgs[k:k + 1], one)
        bp, bq, ap, aq = o2.levels(1)
        assert tuple(l1[k]) == (bp[0, 0], bq[0, 0], ap[0, 0], aq[0, 0]), k


def test_level1_trace_hand_example():
    # levels_aggregate.lob: after its 7 messages level 1 is bid 100x5, ask 101x5
    from golden_format import cases
    c = [c for c in cases() if c.name == "levels_aggregate.lob"][0]
    m = c.message_array()
    o = oracle.Oracle(1, c.capacity, 16)
    l1 = o.process_l1(m, np.array([0, len(m)], np.int64))
    assert tuple(l1[0]) == (100, 2, -1, 0)      # first bid only
    assert tuple(l1[2]) == (100, 5, -1, 0)      # second order at 100 joins the level
    assert tuple(l1[4]) == (100, 5, 103, 1)
    assert tuple(l1[5]) == (100, 5, 101, 5)
    assert tuple(l1[6]) == (100, 5, 101, 5)
