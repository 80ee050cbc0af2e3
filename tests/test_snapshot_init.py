"""Books initialised from a level snapshot (Sec. 5.1.1).

A snapshot lists only price levels and their summed volumes, so each level
becomes ONE order holding the whole volume, with OIDs -9000, -9001, ...
descending.  A cancel or delete whose OID is not live on its side then applies
to the snapshot order resting at the cancel's price.  The paper writes the OID
range as [-inf, -9000] but the cancel condition as OID < -9000; this build
reads both as OID <= -9000 (the first snapshot order is cancellable too).

CPU: hand-worked examples pin the oracle's snapshot initialisation (OID
order, short and out-of-order sides, equal prices) and its cancel rule.  GPU:
lob_init_from_levels against the oracle's own initialisation from the same
level arrays, then streams whose cancels name unknown OIDs at snapshot prices,
in the register-resident (capacity <= 128) and grouped shared-memory
(capacity > 128) book layouts.
"""
import numpy as np
import pytest

import lobgen
import oracle
from engine_harness import assert_same, gpu_outputs, oracle_outputs

BID, ASK = 1, -1


def _msg(rows):
    m = np.zeros(len(rows), dtype=lobgen.MSG_DTYPE)
    for i, (t, s, p, q, oid) in enumerate(rows):
        m[i] = (t, s, p, q, oid, 7, 1000 + i)
    return m


def _hand_snapshot(cap):
    """bids 100 x 5, 99 x 7; asks 101 x 4, 103 x 6 -> OIDs -9000 .. -9003."""
    bk = {k: np.full((1, 2, cap), -1, np.int32) for k in ("price", "qty", "oid", "tid")}
    bk["time_ns"] = np.full((1, 2, cap), -1, np.int64)
    bk["count"] = np.array([[2, 2]], np.int32)
    for s, rows in enumerate(([(100, 5, -9000), (99, 7, -9001)],
                              [(101, 4, -9002), (103, 6, -9003)])):
        for j, (p, q, oid) in enumerate(rows):
            bk["price"][0, s, j], bk["qty"][0, s, j], bk["oid"][0, s, j] = p, q, oid
            bk["tid"][0, s, j], bk["time_ns"][0, s, j] = 0, 0
    return bk


def _levels(o):
    bp, bq, ap, aq = o.levels(4)
    return ([(int(p), int(q)) for p, q in zip(bp[0], bq[0]) if p >= 0],
            [(int(p), int(q)) for p, q in zip(ap[0], aq[0]) if p >= 0])


def test_oracle_snapshot_cancel_by_price_hand_worked():
    cap = 8
    o = oracle.Oracle(1, cap, 16, snapshot_cancels=True)
    o.set_book(_hand_snapshot(cap))
    msgs = _msg([
        (2, BID, 99, 3, 555),    # unknown id at 99: snapshot order -9001 7 -> 4
        (3, ASK, 103, 6, 777),   # delete unknown id at 103: snapshot order -9003 gone
        (2, BID, 98, 1, 888),    # no snapshot order at 98: no-op
        (2, BID, 101, 1, 889),   # 101 is an ask level: the side decides, no-op
        (1, BID, 99, 2, 10),     # a live order joins level 99 behind the snapshot order
        (2, BID, 99, 4, 556),    # unknown id at 99: the snapshot order (4 -> 0) is removed,
        (2, BID, 99, 1, 557),    # ...after which order 10 (positive OID) is never a match
        (2, BID, 99, 1, 10),     # its own id still cancels it: 2 -> 1
        (2, BID, 100, 1, 558),   # OID -9000 itself is a snapshot order: 5 -> 4
    ])
    o.process(msgs, np.array([0, len(msgs)], np.int64))
    bids, asks = _levels(o)
    assert bids == [(100, 4), (99, 1)]
    assert asks == [(101, 4)]
    bk = o.book()
    assert list(bk["oid"][0, 0, :2]) == [-9000, 10]
    assert o.trades()[1][0] == 0


def test_oracle_snapshot_rule_off_by_default():
    cap = 8
    o = oracle.Oracle(1, cap, 16)
    o.set_book(_hand_snapshot(cap))
    msgs = _msg([(2, BID, 99, 3, 555), (3, ASK, 103, 6, 777)])
    o.process(msgs, np.array([0, len(msgs)], np.int64))
    assert _levels(o) == ([(100, 5), (99, 7)], [(101, 4), (103, 6)])


def test_oracle_snapshot_orders_trade_like_any_order():
    # a marketable limit and a market order consume the snapshot orders at
    # their own prices, oldest first (Sec. 4.2); the cancel fallback then
    # finds nothing at the emptied level
    cap = 8
    o = oracle.Oracle(1, cap, 16, snapshot_cancels=True)
    o.set_book(_hand_snapshot(cap))
    msgs = _msg([
        (1, BID, 101, 4, 20),    # takes all of -9002 at 101
        (4, ASK, 0, 6, 21),      # market sell: 5 from -9000 at 100, 1 from -9001 at 99
        (2, ASK, 101, 1, 999),   # level 101 is gone: no-op
    ])
    o.process(msgs, np.array([0, len(msgs)], np.int64))
    tr, cnt = o.trades()
    assert cnt[0] == 3
    t = tr.view(np.int32).reshape(1, 16, 8)[0, :3]
    # trade rows: price, qty, aggressor oid, standing oid, ...
    assert [tuple(int(x) for x in r[:4]) for r in t] == [
        (101, 4, 20, -9002), (100, 5, 21, -9000), (99, 1, 21, -9001)]
    assert _levels(o) == ([(99, 6)], [(103, 6)])


def _levels_case():
    """Three books' level snapshots, depth 3 (int32 [3][3] per array).
    book 0: bids 100x5, 99x7, 98x1; asks 101x4, 103x6, then an empty level
    book 1: bids 50x3, then a level with volume 0 (the side ends there, the
            48x9 after it is not listed); asks 51x2, 52x2, 53x2
    book 2: bids 100x1, 101x1 (out of priority order: the side loads empty but
            its two levels still use OIDs -9000, -9001); asks 102x1, 102x3
            (equal prices: two orders at one level, in listed order)"""
    bp = np.array([[100, 99, 98], [50, 49, 48], [100, 101, -1]], np.int32)
    bq = np.array([[5, 7, 1], [3, 0, 9], [1, 1, 0]], np.int32)
    ap = np.array([[101, 103, -1], [51, 52, 53], [102, 102, -1]], np.int32)
    aq = np.array([[4, 6, 0], [2, 2, 2], [1, 3, 0]], np.int32)
    return bp, bq, ap, aq


# the books the snapshot reading gives, worked out by hand (capacity 4)
HAND_INIT = {
    "count": [[3, 2], [1, 3], [0, 2]],
    "price": [[[100, 99, 98, -1], [101, 103, -1, -1]],
              [[50, -1, -1, -1], [51, 52, 53, -1]],
              [[-1, -1, -1, -1], [102, 102, -1, -1]]],
    "qty": [[[5, 7, 1, -1], [4, 6, -1, -1]],
            [[3, -1, -1, -1], [2, 2, 2, -1]],
            [[-1, -1, -1, -1], [1, 3, -1, -1]]],
    "oid": [[[-9000, -9001, -9002, -1], [-9003, -9004, -1, -1]],
            [[-9000, -1, -1, -1], [-9001, -9002, -9003, -1]],
            [[-1, -1, -1, -1], [-9002, -9003, -1, -1]]],
    "tid": [[[0, 0, 0, -1], [0, 0, -1, -1]],
            [[0, -1, -1, -1], [0, 0, 0, -1]],
            [[-1, -1, -1, -1], [0, 0, -1, -1]]],
    "time_ns": [[[77, 77, 77, -1], [77, 77, -1, -1]],
                [[77, -1, -1, -1], [77, 77, 77, -1]],
                [[-1, -1, -1, -1], [77, 77, -1, -1]]],
}


def test_oracle_init_from_levels_hand_worked():
    o = oracle.Oracle(3, 4, 8)
    assert o.init_from_levels(*_levels_case(), time_ns=77) == 1  # book 2's bid side
    bk = o.book()
    for k, v in HAND_INIT.items():
        assert bk[k].tolist() == v, k
    # the levels of the loaded books read back as the snapshot listed them
    bpx, bqty, apx, aqty = o.levels(3)
    assert bpx[0].tolist() == [100, 99, 98] and bqty[0].tolist() == [5, 7, 1]
    assert apx[2].tolist() == [102, -1, -1] and aqty[2].tolist() == [4, 0, 0]
    assert o.trades()[1].tolist() == [0, 0, 0]


def test_oracle_init_from_levels_then_cancel_by_price():
    # the initialised book equals the hand-built one the cancel-rule example uses
    cap = 8
    bp = np.array([[100, 99]], np.int32)
    bq = np.array([[5, 7]], np.int32)
    ap = np.array([[101, 103]], np.int32)
    aq = np.array([[4, 6]], np.int32)
    o = oracle.Oracle(1, cap, 16, snapshot_cancels=True)
    o.init_from_levels(bp, bq, ap, aq, time_ns=0)
    ref = _hand_snapshot(cap)
    for k, v in o.book().items():
        assert np.array_equal(v, ref[k]), k


def test_oracle_snapshot_cancel_takes_the_earliest_of_equal_price_orders():
    """Two listed levels at one price become two snapshot orders of one level,
    in listed order; a cancel of an unknown id at that price reduces the
    earlier one (its priority is higher), and after it leaves, the later."""
    cap = 8
    o = oracle.Oracle(1, cap, 16, snapshot_cancels=True)
    bp = np.array([[100, 100, 99]], np.int32)
    bq = np.array([[5, 3, 7]], np.int32)
    ap = np.array([[101, 102, 103]], np.int32)
    aq = np.array([[4, 4, 4]], np.int32)
    o.init_from_levels(bp, bq, ap, aq)
    msgs = _msg([
        (2, BID, 100, 2, 555),   # unknown id at 100: the earlier order -9000, 5 -> 3
        (3, BID, 100, 3, 556),   # delete unknown id at 100: -9000 (3 left) leaves
        (2, BID, 100, 1, 557),   # now the later one, -9001: 3 -> 2
    ])
    o.process(msgs, np.array([0, len(msgs)], np.int64))
    bk = o.book()
    assert bk["oid"][0, 0, :2].tolist() == [-9001, -9002]
    assert bk["qty"][0, 0, :2].tolist() == [2, 7]
    assert _levels(o)[0] == [(100, 2), (99, 7)]


def _snapshot_workload(n_books, depth, n_msgs, seed):
    """Seeded level snapshots (10 levels a side, one tick apart around a mid
    price) and per-book streams: lobgen flow with, interleaved, cancels and
    deletes of OIDs that were never submitted, at snapshot prices."""
    rng = np.random.default_rng(seed)
    mid = rng.integers(5_000, 20_000, n_books)
    spread = rng.integers(1, 4, n_books)
    lv = np.arange(depth)
    bid_px = (mid[:, None] - lv[None, :]).astype(np.int32)
    ask_px = (mid[:, None] + spread[:, None] + lv[None, :]).astype(np.int32)
    bid_q = rng.integers(1, 400, (n_books, depth)).astype(np.int32)
    ask_q = rng.integers(1, 400, (n_books, depth)).astype(np.int32)
    # some books list fewer levels on a side
    short = rng.random(n_books) < 0.2
    bid_px[short, depth // 2:] = -1
    bid_q[short, depth // 2:] = 0
    p = lobgen.make_params(seed, "pm1")
    flow, off = lobgen.generate(p, [n_msgs] * n_books)
    parts, offs = [], [0]
    unknown = 1_500_000_000
    for b in range(n_books):
        f = flow[off[b]:off[b + 1]].copy()
        # centre the flow on this book's snapshot
        f["price"] = np.where(f["type"] == 4, f["price"], f["price"] - 10_000 + mid[b])
        k = n_msgs // 5
        snap = np.zeros(k, dtype=lobgen.MSG_DTYPE)
        side = np.where(rng.random(k) < 0.5, BID, ASK)
        j = rng.integers(0, depth, k)
        snap["type"] = np.where(rng.random(k) < 0.5, 2, 3)
        snap["side"] = side
        snap["price"] = np.where(side == BID, bid_px[b, j], ask_px[b, j])
        snap["price"] = np.where(snap["price"] > 0, snap["price"], mid[b])
        snap["qty"] = rng.integers(1, 300, k)
        snap["oid"] = unknown - np.arange(k)
        unknown -= k
        snap["tid"] = 3
        pos = np.sort(rng.integers(0, len(f) + 1, k))
        merged = np.insert(f, pos, snap)
        merged["time_ns"] = np.arange(len(merged))
        parts.append(merged)
        offs.append(offs[-1] + len(merged))
    return (bid_px, bid_q, ask_px, ask_q), np.concatenate(parts), np.array(offs, np.int64)


@pytest.mark.gpu
@pytest.mark.parametrize("cap", [32, 128, 300])
def test_gpu_snapshot_cancels_match_oracle(cap):
    import torch

    import paper_2308_13289_b300 as eng
    n_books, depth, n_msgs = 64, 10, 1500
    (bp, bq, ap, aq), msgs, off = _snapshot_workload(n_books, depth, n_msgs, 4242 + cap)
    tcap = 4096
    t = [torch.from_numpy(x).cuda() for x in (bp, bq, ap, aq)]
    e = eng.Engine(n_books, cap, tcap, snapshot_cancels=True)
    e.init_from_levels(*t, time_ns=0)
    e.process_batch(eng.messages_to_device(msgs), torch.from_numpy(off).cuda())
    g = gpu_outputs(e)
    e.close()
    # the oracle builds its own books from the same level arrays
    o = oracle.Oracle(n_books, cap, tcap, snapshot_cancels=True)
    assert o.init_from_levels(bp, bq, ap, aq, time_ns=0) == 0
    o.process(msgs, off)
    ref = oracle_outputs(o)
    assert_same(g, ref)
    # the workload really exercises the rule: more cancels hit than without it
    off_rule = oracle.Oracle(n_books, cap, tcap)
    off_rule.init_from_levels(bp, bq, ap, aq, time_ns=0)
    off_rule.process(msgs, off)
    hit = oracle.COUNTERS.index("cancel_hit")
    assert ref["counters"][:, hit].sum() > off_rule.counters()[:, hit].sum() + 100


@pytest.mark.gpu
def test_gpu_snapshot_flag_off_ignores_unknown_ids():
    import torch

    import paper_2308_13289_b300 as eng
    n_books, depth, n_msgs, cap, tcap = 32, 10, 800, 64, 2048
    (bp, bq, ap, aq), msgs, off = _snapshot_workload(n_books, depth, n_msgs, 99)
    t = [torch.from_numpy(x).cuda() for x in (bp, bq, ap, aq)]
    e = eng.Engine(n_books, cap, tcap)
    e.init_from_levels(*t)
    e.process_batch(eng.messages_to_device(msgs), torch.from_numpy(off).cuda())
    g = gpu_outputs(e)
    e.close()
    o = oracle.Oracle(n_books, cap, tcap)
    o.init_from_levels(bp, bq, ap, aq)
    o.process(msgs, off)
    assert_same(g, oracle_outputs(o))


def _random_levels(n_books, depth, seed):
    """Level snapshots with every case the reading names: full and short
    sides, empty sides, levels of equal price, sides out of priority order."""
    rng = np.random.default_rng(seed)
    mid = rng.integers(1_000, 50_000, n_books)
    gaps = rng.integers(0, 3, (n_books, depth))  # 0: a level at the previous price
    bp = (mid[:, None] - np.cumsum(gaps, axis=1)).astype(np.int32)
    ap = (mid[:, None] + 1 + np.cumsum(gaps[:, ::-1], axis=1)).astype(np.int32)
    bq = rng.integers(1, 1_000, (n_books, depth)).astype(np.int32)
    aq = rng.integers(1, 1_000, (n_books, depth)).astype(np.int32)
    for arr_p, arr_q in ((bp, bq), (ap, aq)):
        cut = rng.integers(0, depth + 1, n_books)      # listed levels per side
        for b in range(n_books):
            if rng.random() < 0.5:
                arr_p[b, cut[b]:] = np.where(rng.random(depth - cut[b]) < 0.5, -1, 0)
                arr_q[b, cut[b]:] = np.where(arr_p[b, cut[b]:] < 0, 0, rng.integers(0, 9))
    swap = rng.random(n_books) < 0.1                   # out of priority order
    bp[swap, 0], bp[swap, -1] = bp[swap, -1].copy(), bp[swap, 0].copy()
    return bp, bq, ap, aq


@pytest.mark.gpu
@pytest.mark.parametrize("cap,depth", [(7, 7), (32, 10), (100, 10), (128, 64), (300, 40),
                                       (512, 512)])
def test_gpu_init_from_levels_matches_oracle(cap, depth):
    """lob_init_from_levels against the oracle's own snapshot initialisation:
    canonical books, levels and the status bit of sides loaded empty."""
    import torch

    import paper_2308_13289_b300 as eng
    n_books = 96
    bp, bq, ap, aq = _random_levels(n_books, depth, 100 + cap)
    e = eng.Engine(n_books, cap, 16)
    e.init_from_levels(*[torch.from_numpy(x).cuda() for x in (bp, bq, ap, aq)], time_ns=123456789)
    g = gpu_outputs(e)
    _, st = e.stats()
    e.close()
    o = oracle.Oracle(n_books, cap, 16)
    emptied = o.init_from_levels(bp, bq, ap, aq, time_ns=123456789)
    ref = oracle_outputs(o)
    # some sides are listed out of priority order: loaded empty and flagged
    assert emptied > 0
    ref["status"] = eng.STATUS_BAD_BOOK_LOAD
    assert_same(g, ref)
    assert int(st.item()) == eng.STATUS_BAD_BOOK_LOAD


@pytest.mark.gpu
def test_gpu_init_from_levels_rejects_bad_depth():
    import torch

    import paper_2308_13289_b300 as eng
    e = eng.Engine(4, 8, 16)
    z = torch.ones((4, 9), dtype=torch.int32, device="cuda")
    with pytest.raises(eng.LobError):
        e.init_from_levels(z, z, z, z)  # depth 9 > capacity 8
    e.close()


@pytest.mark.gpu
@pytest.mark.parametrize("cap", [32, 100, 300])
def test_gpu_snapshot_cancels_at_equal_price_levels(cap):
    """Snapshots listing several levels at one price (several snapshot orders
    in one level): price-matched cancels take them earliest first, on the GPU
    as in the oracle, in both book layouts."""
    import torch

    import paper_2308_13289_b300 as eng
    n_books, depth, tcap = 48, 12, 1024
    rng = np.random.default_rng(cap)
    mid = rng.integers(1_000, 9_000, n_books)
    # each price listed up to three times in a row
    step = (rng.random((n_books, depth)) < 0.4).astype(np.int64)
    step[:, 0] = 0
    bp = (mid[:, None] - 1 - np.cumsum(step, axis=1)).astype(np.int32)
    ap = (mid[:, None] + 1 + np.cumsum(step, axis=1)).astype(np.int32)
    bq = rng.integers(1, 50, (n_books, depth)).astype(np.int32)
    aq = rng.integers(1, 50, (n_books, depth)).astype(np.int32)
    rows, offs = [], [0]
    for b in range(n_books):
        k = 200
        side = np.where(rng.random(k) < 0.5, BID, ASK)
        lvl = rng.integers(0, depth, k)
        m = np.zeros(k, dtype=lobgen.MSG_DTYPE)
        m["type"] = np.where(rng.random(k) < 0.7, 2, 3)
        m["side"] = side
        m["price"] = np.where(side == BID, bp[b, lvl], ap[b, lvl])
        m["qty"] = rng.integers(1, 30, k)
        m["oid"] = 2_000_000_000 - np.arange(k)
        m["tid"] = 5
        m["time_ns"] = np.arange(k)
        rows.append(m)
        offs.append(offs[-1] + k)
    msgs, off = np.concatenate(rows), np.array(offs, np.int64)
    e = eng.Engine(n_books, cap, tcap, snapshot_cancels=True)
    e.init_from_levels(*[torch.from_numpy(x).cuda() for x in (bp, bq, ap, aq)])
    e.process_batch(eng.messages_to_device(msgs), torch.from_numpy(off).cuda())
    g = gpu_outputs(e)
    e.close()
    o = oracle.Oracle(n_books, cap, tcap, snapshot_cancels=True)
    assert o.init_from_levels(bp, bq, ap, aq) == 0
    o.process(msgs, off)
    ref = oracle_outputs(o)
    assert_same(g, ref)
    # the rule is exercised: about 56 of each book's 200 cancels find a
    # snapshot order before the book's 24 snapshot orders run out
    hit = oracle.COUNTERS.index("cancel_hit")
    assert ref["counters"][:, hit].sum() > n_books * 30
