"""Extreme values: quantities and prices at INT32_MAX, saturating level
totals (reading 15: level quantities saturate at INT32_MAX), matching whose
running standing quantity passes INT32_MAX, cancels larger than any order.

CPU: a hand-worked example pins the oracle.  GPU: the CUDA path against the
oracle on seeded streams of such messages, register-resident (capacity <= 128)
and grouped shared-memory (capacity > 128) books, both full-side rules,
including the level-1 trace and 64-level snapshots.
"""
import numpy as np
import pytest

import lobgen
import oracle
from engine_harness import assert_same, gpu_outputs, oracle_outputs

BID, ASK = 1, -1
MAX = 2**31 - 1


def _msgs(rows):
    m = np.zeros(len(rows), dtype=lobgen.MSG_DTYPE)
    for i, (t, s, p, q, oid) in enumerate(rows):
        m[i] = (t, s, p, q, oid, 9, 10 * i)
    return m


def test_oracle_level_totals_saturate_and_fills_stay_exact():
    o = oracle.Oracle(1, 8, 16)
    m = _msgs([
        (1, BID, 100, MAX, 1),      # three bids of 2^31-1 at one price
        (1, BID, 100, MAX, 2),
        (1, BID, 100, MAX, 3),
        (1, ASK, MAX, MAX, 4),      # an ask at the largest price
        (4, ASK, 0, MAX, 5),        # market sell of 2^31-1 takes order 1 exactly
        (4, BID, 0, 5, 6),          # market buy crosses the max-price ask
        (2, BID, 100, MAX, 2),      # cancel larger than order 2: it leaves
    ])
    o.process(m, np.array([0, len(m)], np.int64))
    bp, bq, ap, aq = o.levels(2)
    assert (bp[0, 0], bq[0, 0]) == (100, MAX)       # only order 3 left: exactly MAX
    assert (ap[0, 0], aq[0, 0]) == (MAX, MAX - 5)
    tr, cnt = o.trades()
    t = tr.view(np.int32).reshape(1, 16, 8)[0]
    assert cnt[0] == 2
    assert tuple(t[0, :4]) == (100, MAX, 5, 1)
    assert tuple(t[1, :4]) == (MAX, 5, 6, 4)
    # before the market sell, the level held 3 * (2^31-1): reported saturated
    o2 = oracle.Oracle(1, 8, 16)
    o2.process(m[:3], np.array([0, 3], np.int64))
    assert o2.levels(1)[1][0, 0] == MAX


def _extreme_streams(n_books, n_msgs, seed):
    """lobgen flow with a third of the quantities replaced by values near
    INT32_MAX, some limit prices at INT32_MAX, and oversized cancels."""
    rng = np.random.default_rng(seed)
    msgs, off = lobgen.generate(lobgen.make_params(seed, "pm1"), [n_msgs] * n_books)
    big = rng.random(len(msgs)) < 0.33
    msgs["qty"] = np.where(big, rng.integers(MAX - 1000, MAX, len(msgs), endpoint=True),
                           msgs["qty"])
    top = (msgs["type"] == 1) & (msgs["side"] == ASK) & (rng.random(len(msgs)) < 0.05)
    msgs["price"] = np.where(top, MAX, msgs["price"])
    return msgs, off


@pytest.mark.gpu
@pytest.mark.parametrize("cap,rule", [(7, 0), (100, 1), (300, 0), (512, 1)])
def test_gpu_extreme_quantities_match_oracle(cap, rule):
    import torch

    import paper_2308_13289_b300 as eng
    msgs, off = _extreme_streams(24, 1500, 77 + cap)
    tcap = 1500
    e = eng.Engine(len(off) - 1, cap, tcap, rule)
    d, doff = eng.messages_to_device(msgs), torch.from_numpy(off).cuda()
    l1 = torch.empty((len(msgs), 4), dtype=torch.int32, device="cuda")
    eng.lob_process_batch_l1(e.h, d, doff, l1)
    g = gpu_outputs(e, depth=64)
    gl1 = l1.cpu().numpy()
    e.close()
    o = oracle.Oracle(len(off) - 1, cap, tcap, rule)
    ol1 = o.process_l1(msgs, off)
    r = oracle_outputs(o, depth=64)
    assert_same(g, r)
    assert np.array_equal(gl1, ol1)
    # the case is really extreme: some level and some level-1 total saturated
    assert (r["bid_qty"] == MAX).any() or (r["ask_qty"] == MAX).any()
    assert (ol1[:, 1] == MAX).any() or (ol1[:, 3] == MAX).any()
