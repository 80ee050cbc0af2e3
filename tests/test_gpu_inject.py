"""Replay, then inject (Sec. 5.1.3 steps 3-4) through the C ABI.

Each step replays a window of data messages on every book with
lob_process_batch (the books' trade logs restart), then submits 1-4 agent
orders to a subset of the books with lob_inject_orders (their trades are
appended to the same logs), then reads the trades and the top levels.  The
oracle processes the same messages in the same order with appended trade logs;
books, trade logs, levels and counters must agree bit for bit after every step,
for register-resident (capacity <= 128) and grouped shared-memory books."""
import numpy as np
import pytest
import torch

import lobgen
import oracle
from engine_harness import assert_same, gpu_outputs, oracle_outputs

pytestmark = pytest.mark.gpu

AGENT_TID = 1_000_000
AGENT_OID0 = 1 << 30


def agent_orders(rng, books, last_ask, step, t_ns):
    """1-4 sells per chosen book: limits at best ask + {-2..+2} ticks or market
    orders, and now and then a marketable buy, so both sides get hit."""
    rows, off = [], [0]
    for i, b in enumerate(books):
        for k in range(int(rng.integers(1, 5))):
            oid = AGENT_OID0 + (step * 64 + i) * 8 + k
            q = int(rng.integers(1, 300))
            kind = rng.random()
            if kind < 0.2:
                rows.append((4, -1, 0, q, oid, AGENT_TID, t_ns[b]))
            elif kind < 0.3:
                rows.append((1, 1, int(last_ask[b]) + int(rng.integers(0, 3)), q, oid, AGENT_TID,
                             t_ns[b]))
            else:
                px = max(1, int(last_ask[b]) + int(rng.integers(-2, 3)))
                rows.append((1, -1, px, q, oid, AGENT_TID, t_ns[b]))
        off.append(len(rows))
    return oracle.messages(rows), np.array(off, np.int64)


@pytest.mark.parametrize("cap", [7, 100, 300])
def test_replay_then_inject_matches_oracle(cap):
    import paper_2308_13289_b300 as eng
    n_books, per, n_steps, tcap = 48, 150, 4, 1024
    rng = np.random.default_rng(cap)
    hs = lobgen.HostStreams(lobgen.make_params(31 + cap), n_books)
    e = eng.Engine(n_books, cap, tcap)
    o = oracle.Oracle(n_books, cap, tcap, append_trades=True)
    for step in range(n_steps):
        m, off = hs.advance([per] * n_books)
        # replay: every book, logs restart
        e.process_batch(eng.messages_to_device(m), torch.from_numpy(off).cuda())
        o.clear_trades()
        o.process(m, off)
        # inject: a different subset of books each step, in a scrambled order
        books = rng.permutation(n_books)[: n_books // 2 + step].astype(np.int32)
        ask_px = o.levels(1)[2][:, 0]
        last_ask = np.where(ask_px > 0, ask_px, 10_000)
        t_ns = m["time_ns"][off[1:] - 1]
        am, aoff = agent_orders(rng, books, last_ask, step, t_ns)
        e.inject_orders(eng.messages_to_device(am), torch.from_numpy(aoff).cuda(),
                        torch.from_numpy(books).cuda())
        o.process(am, aoff, book_ids=books)
        g = gpu_outputs(e)
        ref = oracle_outputs(o)
        assert_same(g, ref)
        # the appended logs really hold agent trades after the replay's
        tr = ref["trades"]
        agent = (tr[..., 4] == AGENT_TID) | (tr[..., 5] == AGENT_TID)
        assert agent.any()


def test_inject_empty_subset_is_a_no_op():
    import paper_2308_13289_b300 as eng
    n_books, cap, tcap = 8, 100, 256
    m, off = lobgen.generate(lobgen.make_params(5), [300] * n_books)
    e = eng.Engine(n_books, cap, tcap)
    e.process_batch(eng.messages_to_device(m), torch.from_numpy(off).cuda())
    before = gpu_outputs(e)
    z = torch.zeros(1, dtype=torch.int64, device="cuda")
    ids = torch.zeros(0, dtype=torch.int32, device="cuda")
    e.inject_orders(eng.messages_to_device(m[:1]), z, ids)
    after = gpu_outputs(e)
    for k in before:
        assert np.array_equal(np.asarray(before[k]), np.asarray(after[k])), k
