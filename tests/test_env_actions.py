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


# ----------------------------------------------------------------------------- GPU parity

AGENT = 1_000_000


def _random_actions(rng, n_steps, n_env):
    """Sizes of every kind the map must handle: whole and fractional, below
    one share, negative, zero, NaN, +-inf, and larger than the task."""
    a = rng.uniform(0.0, 40.0, (n_steps, n_env, 4)).astype(np.float32)
    pick = rng.random((n_steps, n_env, 4))
    a[pick < 0.15] = 0.0
    a[(pick >= 0.15) & (pick < 0.2)] = 0.5
    a[(pick >= 0.2) & (pick < 0.23)] = -3.0
    a[(pick >= 0.23) & (pick < 0.25)] = np.nan
    a[(pick >= 0.25) & (pick < 0.26)] = np.inf
    a[(pick >= 0.26) & (pick < 0.27)] = -np.inf
    a[(pick >= 0.27) & (pick < 0.29)] = 1e9
    a[(pick >= 0.29) & (pick < 0.35)] = np.floor(a[(pick >= 0.29) & (pick < 0.35)])
    return a


def _oracle_episode(m, n_env, n_steps, per, actions, cap, tcap, parent, ticks, tick):
    env = oracle.EnvOracle(n_env, cap, tcap, n_steps=n_steps, parent_qty=parent, agent_tid=AGENT,
                           depth=10, passive_ticks=ticks, tick_size=tick)
    rows = m.reshape(n_env, n_steps, per)
    t_init = rows[:, 0, 0]["time_ns"].astype(np.int64)
    off = np.arange(0, n_env * per + 1, per, dtype=np.int64)
    outs, obs = [], []
    for t in range(n_steps):
        step = np.ascontiguousarray(rows[:, t, :]).reshape(-1)
        reward, lv, fills, tr = env.step(step, off, None, t, l1=True, actions=actions[t])
        outs.append((reward, lv, fills, tr.reshape(n_env, per, 4), env.state()[0]))
        obs.append(env.observe(tr, per, t_init))
    return env, outs, obs


@pytest.mark.gpu
@pytest.mark.parametrize("cap,per,ticks,tick", [(7, 40, 2, 1), (100, 100, 3, 1), (250, 64, 1, 5),
                                                (33, 37, 2, 1)])
def test_gpu_action_steps_and_observations_match_oracle(cap, per, ticks, tick):
    import torch

    import paper_2308_13289_b300 as eng
    from engine_harness import assert_same, gpu_outputs, oracle_outputs
    n_env, n_steps, parent, tcap = 48, 9, 700, 2048
    p = lobgen.make_params(777 + cap)
    m, _ = lobgen.generate(p, [n_steps * per] * n_env)
    if tick > 1:  # the coarse-tick case: every price on the tick grid
        lim = m["type"] != 4
        m["price"] = np.where(lim, m["price"] * tick, m["price"])
    rng = np.random.default_rng(cap)
    actions = _random_actions(rng, n_steps, n_env)
    oenv, oouts, oobs = _oracle_episode(m, n_env, n_steps, per, actions, cap, tcap, parent,
                                        ticks, tick)

    e = eng.Engine(n_env, cap, tcap)
    env = eng.Env(e, n_steps=n_steps, parent_qty=parent, agent_tid=AGENT, depth=10,
                  msgs_per_step=per, passive_ticks=ticks, tick_size=tick)
    d = eng.messages_to_device(m)
    act = torch.from_numpy(actions).cuda()
    out = env.outputs(n_steps)
    l1 = torch.empty((n_steps, n_env, per, 4), dtype=torch.int32, device="cuda")
    stride = n_steps * per
    for t in range(n_steps):  # one step per launch, the observation after each
        env.run(d, stride, t, 1, None, out, row0=t, l1=l1[t:t + 1], actions=act[t:t + 1])
        ob = env.observe(d, stride, l1[t]).cpu().numpy()
        assert ob.tobytes() == oobs[t].tobytes(), "observation differs at step %d: %s" % (
            t, np.argwhere(ob != oobs[t])[:4])
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in out.items()}
    gl1 = l1.cpu().numpy()
    for t in range(n_steps):
        reward, lv, fills, tr, _ = oouts[t]
        assert g["reward"][t].tobytes() == reward.tobytes(), t
        assert np.array_equal(g["fills"][t], fills), t
        for name, v in zip(("bid_px", "bid_qty", "ask_px", "ask_qty"), lv):
            assert np.array_equal(g[name][t], v), (name, t)
        assert np.array_equal(gl1[t], tr), t
    st, p0 = env.state()
    ost, op0 = oenv.state()
    assert np.array_equal(st.cpu().numpy(), ost)
    assert p0.cpu().numpy().tobytes() == op0.tobytes()
    assert_same(gpu_outputs(e), oracle_outputs(oenv.books))
    # the cap was exercised: some tasks were fully placed before the last step
    assert (oouts[n_steps - 2][4][:, 0] == parent).any()
    env.close()
    e.close()


@pytest.mark.gpu
def test_gpu_action_episode_in_one_launch_matches_per_step():
    import torch

    import paper_2308_13289_b300 as eng
    n_env, n_steps, per, cap, parent = 64, 12, 50, 100, 400
    m, _ = lobgen.generate(lobgen.make_params(31337), [n_steps * per] * n_env)
    actions = _random_actions(np.random.default_rng(5), n_steps, n_env)
    act = torch.from_numpy(actions).cuda()
    d = eng.messages_to_device(m)
    res = []
    for splits in ([1] * n_steps, [n_steps], [5, 7]):
        e = eng.Engine(n_env, cap, 1024)
        env = eng.Env(e, n_steps=n_steps, parent_qty=parent, agent_tid=AGENT, msgs_per_step=per)
        out = env.outputs(n_steps)
        t = 0
        for k in splits:
            env.run(d, n_steps * per, t, k, None, out, row0=t, actions=act[t:t + k])
            t += k
        torch.cuda.synchronize()
        st, _ = env.state()
        res.append(({k: v.cpu().numpy() for k, v in out.items()}, st.cpu().numpy()))
        env.close()
        e.close()
    for r in res[1:]:
        for k in r[0]:
            assert r[0][k].tobytes() == res[0][0][k].tobytes(), k
        assert np.array_equal(r[1], res[0][1])


@pytest.mark.gpu
def test_gpu_env_run_needs_exactly_one_agent_source():
    import torch

    import paper_2308_13289_b300 as eng
    e = eng.Engine(4, 16, 64)
    env = eng.Env(e, n_steps=3, msgs_per_step=8)
    d = torch.zeros((4 * 24, 32), dtype=torch.uint8, device="cuda")
    out = env.outputs(1)
    dr = torch.zeros((1, 4), dtype=torch.int32, device="cuda")
    act = torch.zeros((1, 4, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(eng.LobError):
        env.run(d, 24, 0, 1, None, out)
    with pytest.raises(eng.LobError):
        env.run(d, 24, 0, 1, dr, out, actions=act)
    env.close()
    e.close()
