"""Serving loop: continuous batching with admission by HBM footprint.

Each episode's results are the same when it is served alone and inside a mix
where others arrive, wait, run and leave around it (tolerance: exact, all
outputs are integers).  Checked on both paths of the server: the synchronous
one (every tick waited for; per-step levels and trade counts compared) and the
asynchronous one the benchmark runs (the host runs up to RING ticks ahead,
windows are produced on a second stream, staging buffers are reused), where
every episode's final book and counters are compared.  A subset is replayed
step by step through the CPU oracle.  Capacities 7, 100, 250 and 500 cover
register-resident and grouped shared-memory books."""
import copy

import numpy as np
import pytest

import lobgen
import oracle

pytestmark = pytest.mark.gpu

CAPS = (7, 100, 250, 500)
SEED = 77


def _mix(n=40, seed=5, caps=CAPS):
    from paper_2308_13289_b300.serve import Episode
    rng = np.random.default_rng(seed)
    eps = []
    for i in range(n):
        eps.append(Episode(id=1000 + i, capacity=int(rng.choice(caps)),
                           n_steps=int(rng.integers(3, 21)), msgs_per_step=int(rng.integers(20, 61)),
                           arrival=float(rng.integers(0, 30))))
    return eps


def _clone(eps):
    return [copy.copy(e) for e in eps]


def _alone(ep):
    from paper_2308_13289_b300.serve import Server
    srv = Server(capacities=(ep.capacity,), trade_capacity=512, max_slots=1, collect=True,
                 seed=SEED, msgs_per_step=(20, 60))
    e1 = copy.copy(ep)
    e1.arrival = 0.0
    srv.run([e1], clock="virtual")
    return srv


def _oracle_episode(ep):
    """The episode replayed step by step through the CPU oracle: per-step
    (levels, trade count), final book, counters."""
    params = lobgen.make_params(SEED, "pm1")
    hs = lobgen.HostStreams(params, 1, stream_ids=[ep.id])
    o = oracle.Oracle(1, ep.capacity, 512)
    steps = []
    for _ in range(ep.n_steps):
        m, off = hs.advance([ep.msgs_per_step])
        o.process(m, off)
        steps.append((tuple(x[0].tolist() for x in o.levels(10)), int(o.trades()[1][0])))
    return steps, {k: v[0] for k, v in o.book().items()}, o.counters()[0]


def _pick(eps):
    """Episodes of every capacity for the alone / oracle comparisons."""
    out = []
    for c in CAPS:
        out += [e for e in eps if e.capacity == c][:3]
    return out


def test_alone_equals_mix_and_oracle():
    from paper_2308_13289_b300.serve import Server
    eps = _mix()
    srv = Server(capacities=CAPS, trade_capacity=512, max_slots=6, collect=True, seed=SEED,
                 msgs_per_step=(20, 60))
    rep = srv.run(_clone(eps), clock="virtual")
    assert rep["episode_steps"] == sum(e.n_steps for e in eps)
    assert rep["max_queue"] > 0, "the mix should make episodes wait for slots"
    assert rep["max_active"] > 6, "several capacity classes should run at once"
    for ep in _pick(eps):
        alone = _alone(ep)
        assert alone.records[ep.id] == srv.records[ep.id], ep.id
        for k, v in alone.final_books[ep.id].items():
            assert np.array_equal(v, srv.final_books[ep.id][k]), (ep.id, k)
        steps, book, ctr = _oracle_episode(ep)
        assert srv.records[ep.id] == steps, ep.id
        for k, v in book.items():
            assert np.array_equal(v, srv.final_books[ep.id][k]), (ep.id, k)
        assert np.array_equal(srv.final_counters[ep.id], ctr), ep.id


def test_async_run_ahead_equals_alone_and_oracle():
    """The benchmark's path: no tick is waited for, windows come from the
    generator stream, slots are reused as soon as the host sees an episode
    end.  Every episode's final book and counters equal the synchronous
    alone run and the oracle."""
    from paper_2308_13289_b300.serve import RING, Server
    eps = _mix(48, seed=11)
    srv = Server(capacities=CAPS, trade_capacity=512, max_slots=5, keep_final=True, seed=SEED,
                 msgs_per_step=(20, 60))
    rep = srv.run(_clone(eps), clock="virtual")
    assert rep["episode_steps"] == sum(e.n_steps for e in eps)
    assert rep["max_queue"] > 0 and rep["ticks"] > 2 * RING
    assert rep["p50_window_gen_ms"] is not None
    assert set(srv.final_books) == {e.id for e in eps}
    by_id = {e.id: e for e in eps}
    checked = 0
    for ep in _pick(eps):
        alone = _alone(ep)
        for k, v in alone.final_books[ep.id].items():
            assert np.array_equal(v, srv.final_books[ep.id][k]), (ep.id, k)
        assert np.array_equal(alone.final_counters[ep.id], srv.final_counters[ep.id]), ep.id
        checked += 1
    assert checked >= 8
    for eid in sorted(srv.final_books)[::4]:
        _, book, ctr = _oracle_episode(by_id[eid])
        for k, v in book.items():
            assert np.array_equal(v, srv.final_books[eid][k]), (eid, k)
        assert np.array_equal(srv.final_counters[eid], ctr), eid


def test_process_segments_equals_process_batch():
    """Scattered (start, count) segments give the contiguous-offsets result."""
    import torch

    import paper_2308_13289_b300 as eng
    from engine_harness import assert_same, gpu_outputs
    n, per = 10, 700
    m, off = lobgen.generate(lobgen.make_params(11), [per] * n)
    d = eng.messages_to_device(m)
    a = eng.Engine(n, 100, 2048)
    a.process_batch(d, torch.from_numpy(off).cuda())
    b = eng.Engine(n, 100, 2048)
    perm = np.random.default_rng(1).permutation(n).astype(np.int32)
    starts = torch.from_numpy(off[perm]).cuda()
    counts = torch.full((n,), per, dtype=torch.int64, device="cuda")
    eng.lob_process_segments(b.h, d, starts, counts, torch.from_numpy(perm).cuda())
    assert_same(gpu_outputs(b), gpu_outputs(a))


def test_admission_respects_hbm_budget():
    """Equal footprints: a budget of five episodes admits at most five at a
    time, makes the others queue, and still serves every step."""
    from paper_2308_13289_b300.serve import Server, footprint_bytes
    eps = _mix(24, seed=9)
    for e in eps:
        e.capacity, e.msgs_per_step = 100, 40
    fp = footprint_bytes(100, 256, 40)
    srv = Server(capacities=(100,), hbm_budget=5 * fp, trade_capacity=256, max_slots=64, seed=3,
                 msgs_per_step=(40, 40))
    rep = srv.run(eps, clock="virtual")
    assert rep["max_active"] == 5
    assert rep["max_hbm_bytes_admitted"] == 5 * fp
    assert rep["max_queue"] > 0
    assert rep["episode_steps"] == sum(e.n_steps for e in eps)


def test_degenerate_episodes_empty_windows_single_steps_and_slot_reuse():
    """Episodes with empty step windows (0 messages a step), single-step
    episodes and one slot per class, so every slot is reused many times on the
    run-ahead path: every episode's final book and counters equal the oracle
    replaying it (an empty window leaves the book as it was)."""
    from paper_2308_13289_b300.serve import Episode, Server
    rng = np.random.default_rng(21)
    eps = []
    for i in range(30):
        kind = i % 3
        eps.append(Episode(id=5000 + i, capacity=int(rng.choice((7, 250))),
                           n_steps=1 if kind == 0 else int(rng.integers(2, 9)),
                           msgs_per_step=0 if kind == 1 else int(rng.integers(20, 61)),
                           arrival=float(i // 4)))
    srv = Server(capacities=(7, 250), trade_capacity=512, max_slots=1, keep_final=True,
                 seed=SEED, msgs_per_step=(0, 60))
    rep = srv.run(_clone(eps), clock="virtual")
    assert rep["episode_steps"] == sum(e.n_steps for e in eps)
    assert set(srv.final_books) == {e.id for e in eps}
    for ep in eps:
        _, book, ctr = _oracle_episode(ep)
        for k, v in book.items():
            assert np.array_equal(v, srv.final_books[ep.id][k]), (ep.id, k)
        assert np.array_equal(srv.final_counters[ep.id], ctr), ep.id
        if ep.msgs_per_step == 0:
            assert int(srv.final_books[ep.id]["count"].sum()) == 0


def test_window_buckets_route_episodes_and_keep_results():
    """Pools split by messages per step (window_buckets), each ticking at its
    own pace: every episode runs in the pool of its capacity and window
    range, and its final book and counters equal the oracle's and the
    unsplit lockstep server's."""
    from paper_2308_13289_b300.serve import Server
    eps = _mix(36, seed=13)
    runs = {}
    for buckets in ((), (30, 45)):
        # the split pools tick at their own pace (independent scheduling)
        srv = Server(capacities=CAPS, trade_capacity=512, max_slots=4, keep_final=True,
                     seed=SEED, msgs_per_step=(20, 60), window_buckets=buckets,
                     independent=bool(buckets))
        rep = srv.run(_clone(eps), clock="virtual")
        assert rep["episode_steps"] == sum(e.n_steps for e in eps)
        assert len(srv.pools) == len(CAPS) * (len(buckets) + 1)
        for ep in eps:
            p = srv.pool_of(ep)
            assert p.capacity == ep.capacity and ep.msgs_per_step <= p.max_mps
        runs[buckets] = srv
    a, b = runs[()], runs[(30, 45)]
    for ep in eps:
        for k, v in a.final_books[ep.id].items():
            assert np.array_equal(v, b.final_books[ep.id][k]), (ep.id, k)
        assert np.array_equal(a.final_counters[ep.id], b.final_counters[ep.id]), ep.id
    for ep in eps[::5]:
        _, book, ctr = _oracle_episode(ep)
        for k, v in book.items():
            assert np.array_equal(v, b.final_books[ep.id][k]), (ep.id, k)
        assert np.array_equal(b.final_counters[ep.id], ctr), ep.id
