"""Books initialised from a level snapshot (Sec. 5.1.1).

A snapshot lists only price levels and their summed volumes, so each level
becomes ONE order holding the whole volume, with OIDs -9000, -9001, ...
descending.  A cancel or delete whose OID is not live on its side then applies
to the snapshot order resting at the cancel's price.  The paper writes the OID
range as [-inf, -9000] but the cancel condition as OID < -9000; this build
reads both as OID <= -9000 (the first snapshot order is cancellable too).

CPU: a hand-worked example pins the oracle's rule, and the layout that the
package's snapshot helper builds.  GPU: the CUDA path against the oracle on
seeded snapshots plus streams whose cancels name unknown OIDs at snapshot
prices, in the register-resident (capacity <= 128) and grouped shared-memory
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


def test_snapshot_books_layout():
    torch = pytest.importorskip("torch")
    import paper_2308_13289_b300 as eng
    bp = torch.tensor([[100, 99, 98], [50, -1, 48]], dtype=torch.int32)
    bq = torch.tensor([[5, 7, 1], [3, 0, 9]], dtype=torch.int32)
    ap = torch.tensor([[101, 103, -1], [51, 52, 53]], dtype=torch.int32)
    aq = torch.tensor([[4, 6, 0], [2, 2, 2]], dtype=torch.int32)
    bk = eng.snapshot_books(bp, bq, ap, aq, capacity=4, time_ns=77)
    assert bk["count"].tolist() == [[3, 2], [1, 3]]
    assert bk["oid"][0].tolist() == [[-9000, -9001, -9002, -1], [-9003, -9004, -1, -1]]
    assert bk["oid"][1].tolist() == [[-9000, -1, -1, -1], [-9001, -9002, -9003, -1]]
    assert bk["price"][1, 0].tolist() == [50, -1, -1, -1]
    assert bk["qty"][0, 1].tolist() == [4, 6, -1, -1]
    assert bk["time_ns"][0, 0].tolist() == [77, 77, 77, -1]
    assert bk["tid"][1, 1].tolist() == [0, 0, 0, -1]
    with pytest.raises(ValueError):
        eng.snapshot_books(bp, bq, ap, aq, capacity=2)


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
    bk = eng.snapshot_books(*t, capacity=cap, time_ns=0)
    e = eng.Engine(n_books, cap, tcap, snapshot_cancels=True)
    e.set_book(bk)
    e.process_batch(eng.messages_to_device(msgs), torch.from_numpy(off).cuda())
    g = gpu_outputs(e)
    e.close()
    o = oracle.Oracle(n_books, cap, tcap, snapshot_cancels=True)
    o.set_book({k: v.cpu().numpy() for k, v in bk.items()})
    o.process(msgs, off)
    ref = oracle_outputs(o)
    assert_same(g, ref)
    # the workload really exercises the rule: more cancels hit than without it
    off_rule = oracle.Oracle(n_books, cap, tcap)
    off_rule.set_book({k: v.cpu().numpy() for k, v in bk.items()})
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
    bk = eng.snapshot_books(*t, capacity=cap)
    e = eng.Engine(n_books, cap, tcap)
    e.set_book(bk)
    e.process_batch(eng.messages_to_device(msgs), torch.from_numpy(off).cuda())
    g = gpu_outputs(e)
    e.close()
    o = oracle.Oracle(n_books, cap, tcap)
    o.set_book({k: v.cpu().numpy() for k, v in bk.items()})
    o.process(msgs, off)
    assert_same(g, oracle_outputs(o))
