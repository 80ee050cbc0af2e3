"""The CPU oracle (and the paper-literal array version) against the
hand-worked examples in tests/golden/, each derived by hand from Sec. 4.1-4.2."""
import numpy as np
import pytest

import oracle
from golden_format import cases, side_rows, trade_rows

CASES = cases()


@pytest.mark.parametrize("case", CASES, ids=[c.name for c in CASES])
def test_oracle_matches_hand_worked(case):
    m = case.message_array()
    off = np.array([0, len(m)], np.int64)
    o = oracle.Oracle(1, case.capacity, case.trade_capacity, case.rule)
    o.process(m, off)
    bk = o.book()
    assert side_rows(bk, 0, 0) == case.bids
    assert side_rows(bk, 0, 1) == case.asks
    tr, cnt = o.trades()
    assert int(cnt[0]) == case.trades_total
    assert trade_rows(tr, cnt, 0, case.trade_capacity) == case.trades
    # entries past the stored count are all -1
    n_st = min(int(cnt[0]), case.trade_capacity)
    assert (tr[0][n_st:].view(np.int32) == -1).all()
    ctr = dict(zip(oracle.COUNTERS, o.counters()[0]))
    for k, v in case.counters.items():
        assert ctr[k] == v, (k, ctr[k], v)
    if case.depth:
        bp, bq, ap, aq = o.levels(case.depth)
        for k, (p, q) in case.lbid.items():
            assert (bp[0, k], bq[0, k]) == (p, q)
        for k, (p, q) in case.lask.items():
            assert (ap[0, k], aq[0, k]) == (p, q)


@pytest.mark.parametrize("case", CASES, ids=[c.name for c in CASES])
def test_literal_matches_hand_worked(case):
    m = case.message_array()
    off = np.array([0, len(m)], np.int64)
    bk, tr, cnt, ctr = oracle.literal_run(m, off, case.capacity, case.trade_capacity, case.rule)
    assert side_rows(bk, 0, 0) == case.bids
    assert side_rows(bk, 0, 1) == case.asks
    assert int(cnt[0]) == case.trades_total
    assert trade_rows(tr, cnt, 0, case.trade_capacity) == case.trades
    c = dict(zip(oracle.COUNTERS, ctr[0]))
    for k, v in case.counters.items():
        assert c[k] == v, (k, c[k], v)


def test_golden_set_covers_the_rules():
    names = {c.name for c in CASES}
    assert len(CASES) >= 20
    for must in ("fifo_one_level.lob", "walk_three_levels.lob", "overflow_evict.lob",
                 "market_exhausts_side.lob", "cancel_more_than_remaining.lob",
                 "equal_timestamps_fifo.lob", "trade_log_bound.lob", "levels_aggregate.lob"):
        assert must in names
