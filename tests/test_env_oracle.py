"""The execution-environment oracle (Sec. 5) against a hand-worked episode,
and structural properties of the synthetic agent on seeded episodes."""
import os

import numpy as np
import pytest

import lobgen
import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def load_env_fixture(path):
    cfg, steps, final, counters = {}, [], {}, {}
    cur = None
    for raw in open(path):
        line = raw.split("#", 1)[0].strip()
        if not line or line.startswith("cite"):
            continue
        k, *r = line.split()
        if k == "config":
            cfg = {r[i]: int(r[i + 1]) for i in range(0, len(r), 2)}
        elif k == "step":
            cur = dict(step=int(r[0]), draw=int(r[2]), msgs=[], trades=[])
            steps.append(cur)
        elif k == "msg":
            cur["msgs"].append(tuple(int(x) for x in r))
        elif k == "trade":
            cur["trades"].append(tuple(int(x) for x in r))
        elif k == "sums":
            cur["sums"] = tuple(int(x) for x in r)
        elif k == "reward":
            # lambda -> float32 bit pattern written by hand
            cur.setdefault("reward", {})[float(r[0])] = int(r[2], 16)
        elif k in ("lbid", "lask"):
            v = [int(x) for x in r]
            cur[k] = [(v[0], v[1]), (v[2], v[3])]
        elif k == "final":
            final = {r[i]: float(r[i + 1]) for i in range(0, len(r), 2)}
        elif k == "counter":
            counters[r[0]] = int(r[1])
    return cfg, steps, final, counters


ENV_FIXTURES = ["env_three_steps.env", "env_two_steps_mixed.env"]


def reward_bits(x):
    return int(np.asarray(x, dtype=np.float32).view(np.uint32))


@pytest.mark.parametrize("fixture", ENV_FIXTURES)
@pytest.mark.parametrize("lam", [0.0, 0.5])
def test_env_oracle_hand_worked_episode(fixture, lam):
    cfg, steps, final, counters = load_env_fixture(os.path.join(HERE, "golden", fixture))
    env = oracle.EnvOracle(1, cfg["capacity"], 64, n_steps=cfg["n_steps"],
                           parent_qty=cfg["parent"], agent_tid=cfg["agent_tid"],
                           depth=cfg["depth"], p_init_fallback=cfg["p_init_fallback"], lam=lam)
    for st in steps:
        m = oracle.messages(st["msgs"])
        reward, lv, fills = env.step(m, np.array([0, len(m)]), np.array([st["draw"]]), st["step"])
        tr, cnt = env.books.trades()
        got = [tuple(int(x) for x in tr[0][j].tolist()) for j in range(int(cnt[0]))]
        assert got == st["trades"], st["step"]
        sq, spq, aq, apq = st["sums"]
        assert tuple(fills[0]) == (aq, apq)
        # the reward's float32 bits against the value worked out by hand
        assert reward_bits(reward[0]) == st["reward"][lam], (st["step"], float(reward[0]))
        bp, bq, ap, aq_ = lv
        assert [(int(bp[0, k]), int(bq[0, k])) for k in range(2)] == st["lbid"]
        assert [(int(ap[0, k]), int(aq_[0, k])) for k in range(2)] == st["lask"]
    s, p0 = env.state()
    for i, name in enumerate(oracle.EnvOracle.STATE_FIELDS):
        assert s[0, i] == final[name], name
    assert p0[0] == final["p_init"]
    c = dict(zip(oracle.COUNTERS, env.books.counters()[0]))
    for k, v in counters.items():
        assert c[k] == v, k


def test_env_episode_properties():
    """Seeded episodes: the agent never submits before its parent is split, sells
    exactly its parent over the episode when liquidity allows, its orders are
    all sells, and each step's agent fills are part of that step's trades."""
    n_env, n_steps, per = 64, 30, 100
    p = lobgen.make_params(808)
    hs = lobgen.HostStreams(p, n_env)
    draws = lobgen.agent_draws(909, n_env, n_steps)
    env = oracle.EnvOracle(n_env, 100, 20_000, n_steps=n_steps, parent_qty=2000)
    total_fill = np.zeros(n_env, np.int64)
    for t in range(n_steps):
        m, off = hs.advance([per] * n_env)
        reward, lv, fills = env.step(m, off, draws[t], t)
        assert np.isfinite(reward).all()
        total_fill += fills[:, 0]
        tr, cnt = env.books.trades()
        for b in range(0, n_env, 9):
            t_b = tr[b][:cnt[b]]
            agent = (t_b["tid_aggr"] == 1_000_000) | (t_b["tid_stand"] == 1_000_000)
            assert int(t_b["qty"][agent].sum()) == fills[b, 0]
            assert (t_b["tid_stand"][t_b["tid_aggr"] == 1_000_000] != 1_000_000).all()
    s, p0 = env.state()
    assert (s[:, 1] == total_fill).all()
    assert (s[:, 1] <= 2000).all()
    # with deep synthetic books the final market order completes the parent
    assert (s[:, 1] == 2000).mean() > 0.9
    bk = env.books.book()
    assert not (bk["tid"] == 1_000_000).any(), "agent orders left resting after the last step"


def test_env_level1_trace_first_step_equals_book_trace():
    """Before the agent's first order the environment is a plain book: the
    level-1 trace of step 0's data equals the book oracle's trace."""
    p = lobgen.make_params(17)
    m, off = lobgen.generate(p, [100] * 6)
    env = oracle.EnvOracle(6, 100, 512, n_steps=5)
    _, _, _, tr = env.step(m, off, lobgen.agent_draws(1, 6, 1)[0], 0, l1=True)
    o = oracle.Oracle(6, 100, 512)
    assert np.array_equal(tr, o.process_l1(m, off))
