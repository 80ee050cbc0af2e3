"""The paper-literal ablation kernel (lob_literal_process: unsorted arrays,
full scans, optionally every branch of the dispatch on a copy of the book)
against the oracle, bit-exact: canonical books, trade logs and trade counts.
Covers the hand-worked examples, a brute-force corpus of tiny books,
seeded streams at several capacities with ragged and empty segments, both
full-side rules, and both dispatch modes."""
import numpy as np
import pytest
import torch

import lobgen
import oracle
from engine_harness import oracle_outputs
from golden_format import cases

pytestmark = pytest.mark.gpu

KEYS = ("book_price", "book_qty", "book_oid", "book_tid", "book_time_ns", "book_count",
        "trades", "trade_counts")


@pytest.fixture(scope="module")
def eng():
    import paper_2308_13289_b300 as eng
    from paper_2308_13289_b300 import build
    build.build()
    return eng


def _literal(eng, msgs, off, cap, tcap, rule, all_branches):
    bk, tr, cnt = eng.literal_process(eng.messages_to_device(msgs), torch.from_numpy(off).cuda(),
                                      cap, tcap, rule, all_branches)
    torch.cuda.synchronize()
    out = {"book_" + k: v.cpu().numpy() for k, v in bk.items()}
    out["trades"] = tr.cpu().numpy()
    out["trade_counts"] = cnt.cpu().numpy()
    return out


def _oracle(msgs, off, cap, tcap, rule):
    o = oracle.Oracle(len(off) - 1, cap, tcap, rule)
    o.process(msgs, off)
    return oracle_outputs(o)


def _same(g, r):
    for k in KEYS:
        if not np.array_equal(g[k], r[k]):
            d = np.argwhere(g[k] != r[k])
            raise AssertionError("%s differs at %d places, first %s: literal %s oracle %s"
                                 % (k, len(d), d[0], g[k][tuple(d[0])], r[k][tuple(d[0])]))


@pytest.mark.parametrize("all_branches", [False, True])
def test_literal_golden_examples(eng, all_branches):
    for c in cases():
        m = c.message_array()
        off = np.array([0, len(m)], np.int64)
        _same(_literal(eng, m, off, c.capacity, c.trade_capacity, c.rule, all_branches),
              _oracle(m, off, c.capacity, c.trade_capacity, c.rule))


@pytest.mark.parametrize("all_branches", [False, True])
def test_literal_bruteforce_corpus(eng, all_branches):
    from test_oracle_bruteforce import _alphabet, _encode
    alphabet = _alphabet()
    rng = np.random.default_rng(12)
    for cap, rule in ((1, 0), (2, 1), (3, 0), (5, 1)):
        seqs = [tuple(r) for r in rng.integers(0, len(alphabet), size=(5_000, 8))]
        m = _encode(seqs, alphabet)
        off = np.arange(0, len(seqs) * 8 + 1, 8, dtype=np.int64)
        _same(_literal(eng, m, off, cap, 8, rule, all_branches), _oracle(m, off, cap, 8, rule))


@pytest.mark.parametrize("cap,rule", [(1, 0), (7, 1), (33, 0), (64, 0), (100, 0), (100, 1),
                                      (128, 0)])
@pytest.mark.parametrize("all_branches", [False, True])
def test_literal_seeded_streams(eng, cap, rule, all_branches):
    p = lobgen.make_params(2000 + cap, "pm1")
    counts = [1500, 1, 0, 1499, 2049, 64, 65, 300]
    msgs, off = lobgen.generate(p, counts)
    _same(_literal(eng, msgs, off, cap, 1500, rule, all_branches), _oracle(msgs, off, cap, 1500,
                                                                          rule))


def test_literal_equals_engine_and_bounds_trade_log(eng):
    w = lobgen.WORKLOADS["small_16x10k"]
    msgs, off = lobgen.generate(lobgen.make_params(w["seed"], w["mid_walk"]), [3000] * 16)
    tcap = 100  # far below the trades executed: counts keep going, the log stops
    g = _literal(eng, msgs, off, 100, tcap, 0, True)
    e = eng.Engine(16, 100, tcap)
    e.process_batch(eng.messages_to_device(msgs), torch.from_numpy(off).cuda())
    bk = e.book()
    tr, cnt = e.trades()
    torch.cuda.synchronize()
    for k, v in bk.items():
        assert np.array_equal(g["book_" + k], v.cpu().numpy()), k
    assert np.array_equal(g["trades"], tr.cpu().numpy().view(np.int32).reshape(16, tcap, 8))
    assert np.array_equal(g["trade_counts"], cnt.cpu().numpy())
    assert (g["trade_counts"] > tcap).all()
    e.close()


def test_literal_argument_errors(eng):
    m = torch.zeros((8, 8), dtype=torch.int32, device="cuda")
    off = torch.tensor([0, 8], dtype=torch.int64, device="cuda")
    with pytest.raises(eng.LobError):
        eng.literal_process(m, off, 129, 8)  # capacity above 128
    with pytest.raises(eng.LobError):
        eng.literal_process(m, off, 8, 8, overflow_rule=2)
