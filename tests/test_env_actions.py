"""Execution-environment observation vector and four-price action map (Sec. 5.2.2-5.2.3).

Action: four continuous sizes, placed (sell task) at the far touch (best bid),
the mid (rounded up to the tick grid), the near touch (best ask) and the
passive price (best ask + n ticks), in that order; a size is the whole part
of its component, nothing below one share or for NaN, capped by what is left
of the task; an order whose price needs a missing side is not placed.

Observation, float32 [6M + 8]: best bid prices [M], best ask prices [M], mid
prices [M], passive prices [M], spreads [M], current time [s, ns], elapsed
time [s, ns], P_init, drift, task size, executed quantity, imbalances [M].

CPU: hand-worked episodes pin the oracle.  GPU: the CUDA env (actions inside
the fused step kernel, the observation kernel) against the oracle, bit-exact.
"""
import numpy as np
import pytest

import lobgen
import oracle

BID, ASK = 1, -1
T0 = 34_200_000_000_000  # 09:30:00 in ns after midnight


def _msgs(rows):
    m = np.zeros(len(rows), dtype=lobgen.MSG_DTYPE)
    for i, (t, s, p, q, oid, tm) in enumerate(rows):
        m[i] = (t, s, p, q, oid, 5, tm)
    return m


STEP0 = [(1, BID, 100, 5, 1, T0), (1, BID, 98, 10, 2, T0 + 1),
         (1, ASK, 103, 4, 3, T0 + 2), (1, ASK, 105, 6, 4, T0 + 3)]
T1 = 34_261_500_000_777  # 61.5 s + 777 ns later
STEP1 = [(3, BID, 100, 5, 1, T1)] + [(0, 0, 0, 0, 0, T1)] * 3  # delete, then padding


def _one_env(parent, **kw):
    return oracle.EnvOracle(1, 8, 64, n_steps=3, parent_qty=parent, agent_tid=1_000_000,
                            depth=4, p_init_fallback=10_000, passive_ticks=2, tick_size=1, **kw)


def _step(env, rows, action, l1=False):
    m = _msgs(rows)
    return env.step(m, np.array([0, len(m)], np.int64), None, _step.t, threads=1, l1=l1,
                    actions=np.array([action], np.float32))


def test_action_map_hand_worked():
    env = _one_env(100)
    _step.t = 0
    # book after the window: bids 100x5, 98x10; asks 103x4, 105x6 -> P_init 101.5
    reward, lv, fills = _step(env, STEP0, [2.7, 3.0, 0.5, 4.2])
    # far touch 100: 2 sold into bid 100 (order 1, 5 -> 3); mid ceil(101.5) = 102: 3 rest;
    # near 103: 0.5 share -> none; passive 103 + 2 = 105: 4 rest behind order 4
    bp, bq, ap, aq = (x[0] for x in lv)
    assert list(bp[:2]) == [100, 98] and list(bq[:2]) == [3, 10]
    assert list(ap[:3]) == [102, 103, 105] and list(aq[:3]) == [3, 4, 10]
    assert list(fills[0]) == [2, 200]
    assert reward[0] == 0.0  # the agent's own trade is the step's VWAP
    st, p0 = env.state()
    assert st[0, 0] == 9 and st[0, 1] == 2 and st[0, 2] == 3  # submitted, executed, ids used
    assert p0[0] == 101.5

    _step.t = 1
    # the delete removes bid 100 -> best bid 98, best ask 102 (agent), mid 100;
    # NaN places nothing, +inf places everything left (100 - 9 = 91) at 100
    reward, lv, fills, tr = _step(env, STEP1, [np.nan, np.inf, 0.0, 7.0], l1=True)
    bp, bq, ap, aq = (x[0] for x in lv)
    assert ap[0] == 100 and aq[0] == 91 and bp[0] == 98
    assert list(fills[0]) == [0, 0]
    st, _ = env.state()
    assert st[0, 0] == 100 and st[0, 1] == 2
    assert tr.tolist() == [[98, 10, 102, 3]] * 4

    obs = env.observe(tr.reshape(1, 4, 4), 4, np.array([T0], np.int64))[0]
    f = np.float32
    want = np.concatenate([
        [98] * 4, [102] * 4, [100] * 4, [104] * 4, [4] * 4,           # bid, ask, mid, passive, spread
        [34261, f(500000777)], [61, f(500000777)],                     # current, elapsed [s, ns]
        [101.5, 100 - 101.5, 100, 2],                                  # P_init, drift, Q_task, Q_exec
        [3 - 10] * 4,                                                  # imbalance Q_ask - Q_bid
    ]).astype(np.float32)
    assert obs.shape == (6 * 4 + 8,)
    np.testing.assert_array_equal(obs, want)


def test_action_sizes_capped_by_task():
    env = _one_env(5)
    _step.t = 0
    _step(env, STEP0, [2.7, 3.0, 0.5, 4.2])
    st, _ = env.state()
    assert st[0, 0] == 5  # 2 at the far touch, 3 at the mid, nothing left for the passive order
    _step.t = 1
    _, lv, _ = _step(env, [(0, 0, 0, 0, 0, T0 + 9)] * 4, [9.0, 9.0, 9.0, 9.0])
    st, _ = env.state()
    assert st[0, 0] == 5 and st[0, 2] == 2  # the task is fully placed: no new order


def test_action_prices_with_missing_sides_and_coarse_tick():
    # asks empty: far touch = best bid, mid = best bid (one side), near/passive not placed
    env = oracle.EnvOracle(1, 8, 64, n_steps=3, parent_qty=50, depth=2, passive_ticks=3,
                           tick_size=5)
    _step.t = 0
    reward, lv, fills = _step(env, [(1, BID, 500, 4, 1, T0), (1, BID, 490, 4, 2, T0 + 1)],
                              [1.0, 2.0, 3.0, 4.0])
    # far 500: 1 sold (500x4 -> 3); mid = best bid 500: 2 sold (3 -> 1); near/passive: no ask
    bp, bq, ap, aq = (x[0] for x in lv)
    assert list(bp) == [500, 490] and list(bq) == [1, 4] and ap[0] == -1
    assert list(fills[0]) == [3, 1500]
    st, _ = env.state()
    assert st[0, 0] == 3
    # tick 5, bid 490 / ask 505: mid 497.5 rounds up to the grid at 500; passive 505 + 15
    env2 = oracle.EnvOracle(1, 8, 64, n_steps=3, parent_qty=50, depth=3, passive_ticks=3,
                            tick_size=5)
    _, lv, _ = _step(env2, [(1, BID, 490, 4, 1, T0), (1, ASK, 505, 4, 2, T0 + 1)],
                     [0.0, 2.0, 0.0, 3.0])
    bp, bq, ap, aq = (x[0] for x in lv)
    assert list(ap) == [500, 505, 520] and list(aq) == [2, 4, 3]


def test_observation_missing_sides():
    env = _one_env(10)
    tr = np.array([[[100, 5, -1, 0], [-1, 0, 103, 4], [-1, 0, -1, 0]]], np.int32)
    _step.t = 0
    _step(env, [(0, 0, 0, 0, 0, T0 + 5)], [0, 0, 0, 0])  # empty book: P_init = fallback
    obs = env.observe(tr, 3, np.array([T0], np.int64))[0]
    M = 3
    np.testing.assert_array_equal(obs[:M], [100, -1, -1])
    np.testing.assert_array_equal(obs[M:2 * M], [-1, 103, -1])
    np.testing.assert_array_equal(obs[2 * M:3 * M], [100, 103, -1])     # one-sided mid
    np.testing.assert_array_equal(obs[3 * M:4 * M], [-1, 105, -1])      # passive needs the ask
    np.testing.assert_array_equal(obs[4 * M:5 * M], [-1, -1, -1])       # spread needs both
    np.testing.assert_array_equal(obs[5 * M:5 * M + 8], [34200, 5, 0, 5, 10_000, 0, 10, 0])
    np.testing.assert_array_equal(obs[5 * M + 8:], [-5, 4, 0])
