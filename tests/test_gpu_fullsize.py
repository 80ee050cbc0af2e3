"""Parity at the full workload sizes in the launch configuration bench.py
times (autotuned persistent launch), on sampled outputs the oracle computes
book by book from the books' own streams."""
import numpy as np
import pytest
import torch

import lobgen
import oracle
from engine_harness import oracle_outputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    import paper_2308_13289_b300 as eng
    from paper_2308_13289_b300 import build
    build.build()
    return eng


def _sampled(g, books, o):
    ref = oracle_outputs(o)
    for k in ("book_price", "book_qty", "book_oid", "book_tid", "book_time_ns", "book_count",
              "trade_counts", "bid_px", "bid_qty", "ask_px", "ask_qty", "counters"):
        assert np.array_equal(g[k][books], ref[k]), k
    n_tr = min(4, len(books))
    assert np.array_equal(g["trades"][books[:n_tr]], ref["trades"][:n_tr])


def test_replay_1024x100k_full_size(eng, tmp_path, monkeypatch):
    from engine_harness import gpu_outputs
    from paper_2308_13289_b300 import autotune
    monkeypatch.setenv(autotune.CACHE_ENV, str(tmp_path / "tune.json"))
    w = lobgen.WORKLOADS["replay_1024x100k"]
    n, per = w["n_books"], w["msgs"]
    params = lobgen.make_params(w["seed"], w["mid_walk"])
    dm, doff = lobgen.DeviceStreams(params, n).advance([per] * n)
    tcap = int(per * 0.75) + 1024
    e = eng.Engine(n, w["capacity"], tcap)
    pre = dm.view(n, per, 8)[:, :5000].contiguous().view(-1, 8)
    pre_off = torch.arange(0, n * 5000 + 1, 5000, dtype=torch.int64, device="cuda")
    autotune.apply(e, autotune.tune(n, w["capacity"], pre, pre_off, trade_capacity=5000,
                                    mean_msgs=per, reps=1))
    e.process_batch(dm, doff)
    g = gpu_outputs(e)
    assert g["status"] == 0
    books = np.array([0, 1, 2, 100, 511, 512, 900, 1022, 1023])
    hm, hoff = lobgen.generate(params, [per] * len(books), stream_ids=books.astype(np.uint64))
    o = oracle.Oracle(len(books), w["capacity"], tcap)
    o.process(hm, hoff)
    _sampled(g, books, o)
    # the plain form: one launch per 100-message chunk, trades appended
    chunk = w["chunk"]
    nch = per // chunk
    cm = torch.empty_like(dm)
    cm.view(nch, n, chunk, 8).copy_(dm.view(n, nch, chunk, 8).transpose(0, 1))
    del pre
    ep = eng.Engine(n, w["capacity"], tcap, append_trades=True)
    seg = torch.arange(0, n * chunk + 1, chunk, dtype=torch.int64, device="cuda")
    for c in range(nch):
        ep.process_batch(cm[c * n * chunk:(c + 1) * n * chunk], seg)
    gp = gpu_outputs(ep)
    for k in g:
        if k != "status":
            assert np.array_equal(gp[k], g[k]), k


def test_uneven_4096_full_size_longest_first(eng):
    from engine_harness import gpu_outputs
    w = lobgen.WORKLOADS["uneven_4096_lognormal"]
    n = w["n_books"]
    counts = lobgen.lognormal_counts(n, w["seed"])
    params = lobgen.make_params(w["seed"], w["mid_walk"])
    perm = np.argsort(-counts, kind="stable")
    dm, doff = lobgen.DeviceStreams(params, n).advance(counts[perm], ids=perm.astype(np.int32))
    tcap = int(counts.max() * 0.75) + 1024
    e = eng.Engine(n, w["capacity"], tcap)
    e.process_batch(dm, doff, torch.from_numpy(perm.astype(np.int32)).cuda())
    g = gpu_outputs(e)
    assert g["status"] == 0
    books = np.array(sorted({0, 1, int(perm[0]), int(perm[1]), int(perm[-1]), 2047, 4095}))
    hm, hoff = lobgen.generate(params, counts[books], stream_ids=books.astype(np.uint64))
    o = oracle.Oracle(len(books), w["capacity"], tcap)
    o.process(hm, hoff)
    _sampled(g, books, o)


def test_rl_exec_8192x400_full_size(eng):
    w = lobgen.WORKLOADS["rl_exec_8192x400"]
    n, steps, per = w["n_books"], w["steps"], w["msgs_per_step"]
    params = lobgen.make_params(w["seed"], w["mid_walk"])
    dm, _ = lobgen.DeviceStreams(params, n).advance([steps * per] * n)
    draws = lobgen.agent_draws_device(w["seed"] + 1, n, steps)
    e = eng.Engine(n, w["capacity"], 4096)
    env = eng.Env(e, n_steps=steps, msgs_per_step=per)
    out = env.run(dm, steps * per, 0, steps, draws)
    torch.cuda.synchronize()
    sample = np.array([0, 4097, n - 1])
    hm, _ = lobgen.generate(params, [steps * per] * len(sample), stream_ids=sample.astype(np.uint64))
    hd = lobgen.agent_draws(w["seed"] + 1, n, steps)[:, sample]
    oenv = oracle.EnvOracle(len(sample), w["capacity"], 4096, n_steps=steps)
    rows = hm.reshape(len(sample), steps, per)
    g = {k: v.cpu().numpy() for k, v in out.items()}
    for t in range(steps):
        stp = np.ascontiguousarray(rows[:, t, :]).reshape(-1)
        r_, lv, f_ = oenv.step(stp, np.arange(0, len(sample) * per + 1, per), hd[t], t)
        assert g["reward"][t, sample].tobytes() == r_.tobytes(), t
        assert np.array_equal(g["fills"][t, sample], f_), t
        for name, v in zip(("bid_px", "bid_qty", "ask_px", "ask_qty"), lv):
            assert np.array_equal(g[name][t, sample], v), (name, t)
    st, p0 = env.state()
    ost, op0 = oenv.state()
    assert np.array_equal(st.cpu().numpy()[sample], ost)
    assert p0.cpu().numpy()[sample].tobytes() == op0.tobytes()


def test_replay_1024x100k_invariants_on_every_book(eng):
    """Properties that hold at any size, checked on all 1,024 books and on
    every one of the 1.024e8 level-1 trace rows (the oracle would take
    minutes for all of them): quantity conservation per book, sides in
    priority order with positive quantities and unique ids, no crossed book
    after any message, trade-log totals equal to the traded quantity, and the
    last trace row equal to the top level."""
    w = lobgen.WORKLOADS["replay_1024x100k"]
    _invariants_on_every_book(eng, w["n_books"], w["msgs"], w["capacity"], w["seed"],
                              w["mid_walk"])


@pytest.mark.parametrize("cap", [250, 500])
def test_grouped_books_invariants_on_every_book(eng, cap):
    """The same properties for books kept in shared memory (stored worst
    first), 1,024 books x 2e4 messages."""
    _invariants_on_every_book(eng, 1024, 20_000, cap, 4040 + cap, "pm1")


def _invariants_on_every_book(eng, n, per, cap, seed, walk):
    params = lobgen.make_params(seed, walk)
    dm, doff = lobgen.DeviceStreams(params, n).advance([per] * n)
    tcap = int(per * 0.75) + 1024
    e = eng.Engine(n, cap, tcap)
    l1 = torch.empty((n * per, 4), dtype=torch.int32, device="cuda")
    eng.lob_process_batch_l1(e.h, dm, doff, l1)
    bk = e.book()
    tr, tcnt = e.trades()
    ctr, st = e.stats()
    bp, bq, ap, aq = e.levels(1)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    c = {k: ctr[:, i] for i, k in enumerate(eng.COUNTERS)}
    # conservation: submitted = 2 x traded + cancelled + rejected + evicted + resting + dropped
    live = torch.arange(cap, device="cuda")[None, None, :] < bk["count"][:, :, None].long()
    resting = torch.where(live, bk["qty"].long(), torch.zeros_like(bk["qty"].long())).sum((1, 2))
    lhs = c["limit_qty"] + c["market_qty"]
    rhs = (2 * c["traded_qty"] + c["cancelled_qty"] + c["rejected_qty"] + c["evicted_qty"]
           + resting + c["market_discarded_qty"])
    assert torch.equal(lhs, rhs)
    assert int(c["msgs"].sum()) == n * per
    # sides: priority order, positive quantities, unique ids
    px = bk["price"].long()
    nxt_ok = torch.where(live[:, :, 1:], torch.stack([px[:, 0, :-1] >= px[:, 0, 1:],
                                                      px[:, 1, :-1] <= px[:, 1, 1:]], 1),
                         torch.ones_like(live[:, :, 1:]))
    assert bool(nxt_ok.all())
    assert bool(torch.where(live, bk["qty"] > 0, torch.ones_like(live)).all())
    oid = torch.where(live, bk["oid"].long(), -1 - torch.arange(n * 2 * cap, device="cuda")
                      .view(n, 2, cap))
    assert torch.sort(oid.view(n, -1), 1).values.diff(dim=1).ne(0).all()
    # never crossed, after any message of any book
    both = (l1[:, 0] > 0) & (l1[:, 2] > 0)
    assert bool((l1[:, 0][both] < l1[:, 2][both]).all())
    assert bool(((l1[:, 0] > 0) == (l1[:, 1] > 0)).all())
    last = l1.view(n, per, 4)[:, -1]
    assert torch.equal(last[:, 0], bp[:, 0]) and torch.equal(last[:, 1], bq[:, 0])
    assert torch.equal(last[:, 2], ap[:, 0]) and torch.equal(last[:, 3], aq[:, 0])
    # every trade stored (the log holds them all here) and the totals agree
    assert bool((tcnt <= tcap).all()) and torch.equal(tcnt, c["trades"])
    stored = torch.arange(tcap, device="cuda")[None, :] < tcnt[:, None]
    qty = tr[:, :, 1].long()
    assert bool(torch.where(stored, qty > 0, torch.ones_like(stored)).all())
    assert torch.equal(torch.where(stored, qty, torch.zeros_like(qty)).sum(1), c["traded_qty"])
    e.close()
