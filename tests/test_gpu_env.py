"""Execution-environment steps on the GPU (lob_env_run) vs the environment
oracle, bit-exact: per-step rewards (float32 bits), agent fills, top levels,
final books, trade logs, counters and agent state.  Covers one launch per
step, one persistent launch for a whole episode, a split episode, CUDA-graph
capture of the per-step loop, and several capacities."""
import os

import numpy as np
import pytest
import torch

import lobgen
import oracle
from engine_harness import assert_same, gpu_outputs, oracle_outputs
from test_env_oracle import ENV_FIXTURES, load_env_fixture, reward_bits

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
AGENT = 1_000_000


@pytest.fixture(scope="module")
def eng():
    import paper_2308_13289_b300 as eng
    from paper_2308_13289_b300 import build
    build.build()
    return eng


def episode_streams(n_env, n_steps, per, seed):
    p = lobgen.make_params(seed)
    m, off = lobgen.generate(p, [n_steps * per] * n_env)
    return m, off


def run_oracle(m, n_env, n_steps, per, draws, cap, tcap, lam, depth=10, parent=2000):
    env = oracle.EnvOracle(n_env, cap, tcap, n_steps=n_steps, parent_qty=parent, agent_tid=AGENT,
                           depth=depth, lam=lam)
    rows = m.reshape(n_env, n_steps, per)
    outs = []
    for t in range(n_steps):
        step = np.ascontiguousarray(rows[:, t, :]).reshape(-1)
        off = np.arange(0, n_env * per + 1, per, dtype=np.int64)
        outs.append(env.step(step, off, draws[t], t))
    return env, outs


def run_gpu(eng, m, n_env, n_steps, per, draws, cap, tcap, lam, splits, depth=10, parent=2000,
            graph=False):
    e = eng.Engine(n_env, cap, tcap)
    env = eng.Env(e, n_steps=n_steps, parent_qty=parent, agent_tid=AGENT, depth=depth,
                  msgs_per_step=per, lam=lam)
    d = eng.messages_to_device(m)
    dr = torch.from_numpy(draws.view(np.int32)).cuda()
    out = env.outputs(n_steps)
    if graph:
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                for t in range(n_steps):
                    env.run(d, n_steps * per, t, 1, dr[t:t + 1], out, row0=t)
        torch.cuda.current_stream().wait_stream(s)
        g.replay()
    else:
        t = 0
        for k in splits:
            env.run(d, n_steps * per, t, k, dr[t:t + k], out, row0=t)
            t += k
        assert t == n_steps
    torch.cuda.synchronize()
    return e, env, {k: v.cpu().numpy() for k, v in out.items()}


def compare(e, env, gout, oenv, oouts, n_steps):
    for t in range(n_steps):
        reward, lv, fills = oouts[t]
        assert gout["reward"][t].tobytes() == reward.tobytes(), "reward differs at step %d" % t
        assert np.array_equal(gout["fills"][t], fills), t
        for name, v in zip(("bid_px", "bid_qty", "ask_px", "ask_qty"), lv):
            assert np.array_equal(gout[name][t], v), (name, t)
    st, p0 = env.state()
    ost, op0 = oenv.state()
    assert np.array_equal(st.cpu().numpy(), ost)
    assert p0.cpu().numpy().tobytes() == op0.tobytes()
    assert_same(gpu_outputs(e), oracle_outputs(oenv.books))


@pytest.mark.parametrize("fixture", ENV_FIXTURES)
def test_hand_worked_episode_on_gpu(eng, fixture):
    cfg, steps, final, _ = load_env_fixture(os.path.join(HERE, "golden", fixture))
    per = max(len(s["msgs"]) for s in steps)
    rows = []
    for s in steps:  # pad each window at its front with type-0 messages
        pad = [(0, 0, 0, 0, 0, 0, 0)] * (per - len(s["msgs"]))
        rows += pad + s["msgs"]
    m = oracle.messages(rows)
    draws = np.array([[s["draw"]] for s in steps], dtype=np.uint32)
    for lam in (0.0, 0.5):
        e = eng.Engine(1, cfg["capacity"], 64)
        env = eng.Env(e, n_steps=cfg["n_steps"], parent_qty=cfg["parent"], agent_tid=cfg["agent_tid"],
                      depth=cfg["depth"], p_init_fallback=cfg["p_init_fallback"], msgs_per_step=per,
                      lam=lam)
        oenv = oracle.EnvOracle(1, cfg["capacity"], 64, n_steps=cfg["n_steps"],
                                parent_qty=cfg["parent"], agent_tid=cfg["agent_tid"],
                                depth=cfg["depth"], p_init_fallback=cfg["p_init_fallback"], lam=lam)
        oouts = [oenv.step(m[t * per:(t + 1) * per], np.array([0, per]), draws[t], t)
                 for t in range(cfg["n_steps"])]
        out = env.outputs(cfg["n_steps"])
        env.run(eng.messages_to_device(m), cfg["n_steps"] * per, 0, cfg["n_steps"],
                torch.from_numpy(draws.view(np.int32)).cuda(), out)
        torch.cuda.synchronize()
        g = {k: v.cpu().numpy() for k, v in out.items()}
        compare(e, env, g, oenv, oouts, cfg["n_steps"])
        # and the hand-worked sums and rewards themselves
        for t, s in enumerate(steps):
            assert tuple(g["fills"][t][0]) == s["sums"][2:]
            assert reward_bits(g["reward"][t][0]) == s["reward"][lam], (t, lam)


@pytest.mark.parametrize("splits,lam", [([1] * 40, 0.0), ([40], 0.25), ([17, 23], 0.0)])
def test_seeded_episodes_match_oracle(eng, splits, lam):
    n_env, n_steps, per = 96, 40, 100
    m, _ = episode_streams(n_env, n_steps, per, 4242)
    draws = lobgen.agent_draws(77, n_env, n_steps)
    e, env, g = run_gpu(eng, m, n_env, n_steps, per, draws, 100, 4096, lam, splits)
    oenv, oouts = run_oracle(m, n_env, n_steps, per, draws, 100, 4096, lam)
    compare(e, env, g, oenv, oouts, n_steps)


@pytest.mark.parametrize("cap", [7, 250, 500])
def test_episode_capacities(eng, cap):
    n_env, n_steps, per = 24, 12, 60
    m, _ = episode_streams(n_env, n_steps, per, 99 + cap)
    draws = lobgen.agent_draws(5, n_env, n_steps)
    e, env, g = run_gpu(eng, m, n_env, n_steps, per, draws, cap, 2048, 0.0, [5, 7], parent=600)
    oenv, oouts = run_oracle(m, n_env, n_steps, per, draws, cap, 2048, 0.0, parent=600)
    compare(e, env, g, oenv, oouts, n_steps)


def test_graph_captured_steps_equal_direct(eng):
    n_env, n_steps, per = 64, 20, 100
    m, _ = episode_streams(n_env, n_steps, per, 31)
    draws = lobgen.agent_draws(32, n_env, n_steps)
    e, env, g = run_gpu(eng, m, n_env, n_steps, per, draws, 100, 4096, 0.0, None, graph=True)
    oenv, oouts = run_oracle(m, n_env, n_steps, per, draws, 100, 4096, 0.0)
    compare(e, env, g, oenv, oouts, n_steps)


def test_env_argument_errors(eng):
    e = eng.Engine(4, 100, 64)
    env = eng.Env(e, n_steps=5, msgs_per_step=10)
    d = torch.zeros((4 * 50, 8), dtype=torch.int32, device="cuda")
    dr = torch.zeros((5, 4), dtype=torch.int32, device="cuda")
    with pytest.raises(eng.LobError):
        env.run(d, 50, 3, 3, dr[:3])  # runs past the episode
    with pytest.raises(eng.LobError):
        env.run(d, 10, 0, 1, dr[:1])  # stride shorter than an episode


@pytest.mark.parametrize("cap", [100, 500])
def test_env_level1_trace_matches_oracle(eng, cap):
    n_env, n_steps, per = 32, 8, 50
    m, _ = episode_streams(n_env, n_steps, per, 777 + cap)
    draws = lobgen.agent_draws(8, n_env, n_steps)
    e = eng.Engine(n_env, cap, 2048)
    env = eng.Env(e, n_steps=n_steps, msgs_per_step=per, parent_qty=300)
    l1 = torch.full((n_steps, n_env, per, 4), -7, dtype=torch.int32, device="cuda")
    out = env.run(eng.messages_to_device(m), n_steps * per, 0, n_steps,
                  torch.from_numpy(draws.view(np.int32)).cuda(), l1=l1)
    torch.cuda.synchronize()
    oenv = oracle.EnvOracle(n_env, cap, 2048, n_steps=n_steps, parent_qty=300)
    rows = m.reshape(n_env, n_steps, per)
    g = l1.cpu().numpy()
    for t in range(n_steps):
        stp = np.ascontiguousarray(rows[:, t, :]).reshape(-1)
        r_, lv, f_, tr = oenv.step(stp, np.arange(0, n_env * per + 1, per), draws[t], t, l1=True)
        assert np.array_equal(g[t].reshape(-1, 4), tr), t
        assert out["reward"][t].cpu().numpy().tobytes() == r_.tobytes()


@pytest.mark.parametrize("cap,n_env", [(100, 3000), (250, 3000)])
def test_segmented_persistent_episode_equals_per_step(eng, cap, n_env):
    """More environments than resident warps: the persistent launch hands out
    segments of each episode (each resuming from what the previous one wrote
    back).  Its results equal one launch per step and the oracle, also when
    the same launch runs again and when it is replayed from a CUDA graph
    (whose arguments never change: the segment flags carry a device epoch)."""
    n_steps, per, tcap = 48, 20, 256
    m, _ = episode_streams(n_env, n_steps, per, 515 + cap)
    draws = lobgen.agent_draws(77, n_env, n_steps)
    d = eng.messages_to_device(m)
    dr = torch.from_numpy(draws.view(np.int32)).cuda()

    def make():
        e = eng.Engine(n_env, cap, tcap)
        env = eng.Env(e, n_steps=n_steps, parent_qty=2000, agent_tid=AGENT, msgs_per_step=per)
        return e, env, env.outputs(n_steps)

    def snap(e, env, out):
        torch.cuda.synchronize()
        st, p0 = env.state()
        o = {k: v.cpu().numpy().copy() for k, v in out.items()}
        o["state"], o["p_init"] = st.cpu().numpy(), p0.cpu().numpy()
        o.update({"book_" + k: v.cpu().numpy() for k, v in e.book().items()})
        o["counters"] = e.stats()[0].cpu().numpy()
        return o

    # reference: one launch per step
    e1, env1, out1 = make()
    for t in range(n_steps):
        env1.run(d, n_steps * per, t, 1, dr[t:t + 1], out1, row0=t)
    ref = snap(e1, env1, out1)
    assert env1.segments() == 1
    # one persistent launch, twice on the same objects
    e2, env2, out2 = make()
    for rep in range(2):
        e2.reset()
        env2.reset()
        env2.run(d, n_steps * per, 0, n_steps, dr, out2)
        assert env2.segments() > 1, "the launch should split the episodes"
        got = snap(e2, env2, out2)
        for k, v in ref.items():
            assert v.tobytes() == got[k].tobytes(), (rep, k)
    # the persistent launch captured in a CUDA graph and replayed twice
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            e2.reset()
            env2.reset()
            env2.run(d, n_steps * per, 0, n_steps, dr, out2)
    torch.cuda.current_stream().wait_stream(s)
    for rep in range(2):
        g.replay()
        got = snap(e2, env2, out2)
        for k, v in ref.items():
            assert v.tobytes() == got[k].tobytes(), ("graph", rep, k)
    assert int(e2.stats()[1].item()) == 0
    # and the oracle on a few environments
    sample = np.array([0, 1, n_env // 2, n_env - 1])
    oenv, oouts = run_oracle(m.reshape(n_env, -1)[sample].reshape(-1), len(sample), n_steps, per,
                             draws[:, sample], cap, tcap, 0.0)
    for t in range(n_steps):
        reward, lv, fills = oouts[t]
        assert ref["reward"][t][sample].tobytes() == reward.tobytes(), t
        assert np.array_equal(ref["fills"][t][sample], fills), t
        assert np.array_equal(ref["bid_px"][t][sample], lv[0]), t
    ob = oenv.books.book()
    for k, v in ob.items():
        assert np.array_equal(ref["book_" + k][sample], v), k
