"""Serving loop: continuous batching with admission by HBM footprint.

Each episode's per-step outputs (top levels, trade counts) and final book are
the same when it is served alone and inside a mix where others arrive, wait,
run and leave around it (tolerance: exact, all outputs are integers); a subset
is also replayed step by step through the CPU oracle."""
import numpy as np
import pytest

import lobgen
import oracle

pytestmark = pytest.mark.gpu


def _mix(n=36, seed=5):
    from paper_2308_13289_b300.serve import Episode
    rng = np.random.default_rng(seed)
    eps = []
    for i in range(n):
        eps.append(Episode(id=1000 + i, capacity=int(rng.choice([7, 100, 250])),
                           n_steps=int(rng.integers(3, 21)), msgs_per_step=int(rng.integers(20, 61)),
                           arrival=float(rng.integers(0, 30))))
    return eps


def _clone(eps):
    import copy
    return [copy.copy(e) for e in eps]


def test_alone_equals_mix_and_oracle():
    from paper_2308_13289_b300.serve import Server
    eps = _mix()
    srv = Server(capacities=(7, 100, 250), trade_capacity=512, max_slots=6, collect=True,
                 seed=77)
    rep = srv.run(_clone(eps), clock="virtual")
    assert rep["episode_steps"] == sum(e.n_steps for e in eps)
    assert rep["max_queue"] > 0, "the mix should make episodes wait for slots"
    assert rep["max_active"] > 6, "several capacity classes should run at once"
    for ep in eps[:12]:
        alone = Server(capacities=(ep.capacity,), trade_capacity=512, max_slots=1, collect=True,
                       seed=77)
        import copy
        e1 = copy.copy(ep)
        e1.arrival = 0.0
        alone.run([e1], clock="virtual")
        assert alone.records[ep.id] == srv.records[ep.id], ep.id
        for k, v in alone.final_books[ep.id].items():
            assert np.array_equal(v, srv.final_books[ep.id][k]), (ep.id, k)
    # oracle replay of a few episodes, step by step
    params = lobgen.make_params(77, "pm1")
    for ep in eps[:8]:
        hs = lobgen.HostStreams(params, 1, stream_ids=[ep.id])
        o = oracle.Oracle(1, ep.capacity, 512)
        for t in range(ep.n_steps):
            m, off = hs.advance([ep.msgs_per_step])
            o.process(m, off)
            lv = o.levels(10)
            got_lv, got_tc = srv.records[ep.id][t]
            assert tuple(x[0].tolist() for x in lv) == got_lv, (ep.id, t)
            assert int(o.trades()[1][0]) == got_tc
        ob = o.book()
        for k, v in ob.items():
            assert np.array_equal(v[0], srv.final_books[ep.id][k]), (ep.id, k)


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
    from paper_2308_13289_b300.serve import Server, footprint_bytes
    eps = _mix(24, seed=9)
    for e in eps:
        e.capacity = 100
    fp = footprint_bytes(100, 256)
    srv = Server(capacities=(100,), hbm_budget=5 * fp, trade_capacity=256, max_slots=64, seed=3)
    rep = srv.run(eps, clock="virtual")
    assert rep["max_active"] <= 5
    assert rep["max_hbm_bytes_admitted"] <= 5 * fp
    assert rep["episode_steps"] == sum(e.n_steps for e in eps)
