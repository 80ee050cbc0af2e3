"""CUDA engine vs the CPU oracle, element by element, bit-exact.

Covers the hand-worked examples, a brute-force corpus of tiny books, seeded
streams of the paper-style workloads across capacities (K = 1..16 slots per
lane), both full-side rules, several launch shapes (warps per CTA, staged
chunk sizes), chunked calls, book subsets, ragged and empty segments, and the
device status word."""
import numpy as np
import pytest
import torch

import lobgen
import oracle
from engine_harness import assert_same, gpu_outputs, oracle_outputs, run_both
from golden_format import cases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    import paper_2308_13289_b300 as eng
    from paper_2308_13289_b300 import build
    build.build()
    return eng


def test_golden_examples_on_gpu(eng):
    for c in cases():
        m = c.message_array()
        off = np.array([0, len(m)], np.int64)
        g, r = run_both(m, off, c.capacity, c.trade_capacity, c.rule)
        assert_same(g, r)


def test_bruteforce_corpus_on_gpu(eng):
    from test_oracle_bruteforce import _alphabet, _encode
    alphabet = _alphabet()
    rng = np.random.default_rng(11)
    for cap, rule in ((1, 0), (2, 0), (3, 1), (5, 0)):
        seqs = [tuple(r) for r in rng.integers(0, len(alphabet), size=(20_000, 8))]
        m = _encode(seqs, alphabet)
        off = np.arange(0, len(seqs) * 8 + 1, 8, dtype=np.int64)
        g, r = run_both(m, off, cap, 8, rule)
        assert_same(g, r)


@pytest.mark.parametrize("cap", [1, 7, 33, 100, 128, 250, 500, 512])
def test_seeded_streams_across_capacities(eng, cap):
    p = lobgen.make_params(1000 + cap, "pm1")
    counts = [3000, 1, 0, 2999, 4097, 64, 65, 500]
    msgs, off = lobgen.generate(p, counts)
    g, r = run_both(msgs, off, cap, 3000, 0, depth=12)
    assert_same(g, r)


def test_small_workload_reject_rule(eng):
    w = lobgen.WORKLOADS["small_16x10k"]
    msgs, off = lobgen.generate(lobgen.make_params(w["seed"], w["mid_walk"]), [w["msgs"]] * 16)
    g, r = run_both(msgs, off, 100, 8192, 1)
    assert_same(g, r)


@pytest.mark.parametrize("launch", [(1, 8, 0), (4, 64, 0), (8, 64, 0), (2, 1024, 1), (3, 40, 2)])
def test_launch_shapes(eng, launch):
    w = lobgen.WORKLOADS["small_16x10k"]
    msgs, off = lobgen.generate(lobgen.make_params(w["seed"], w["mid_walk"]), [w["msgs"]] * 16)
    g, r = run_both(msgs, off, 100, 8192, 0, launch=launch)
    assert_same(g, r)


def test_trade_log_bound_counts_dropped(eng):
    msgs, off = lobgen.generate(lobgen.make_params(5), [4000] * 6)
    g, r = run_both(msgs, off, 100, 50, 0)
    assert_same(g, r)
    assert (r["counters"][:, oracle.COUNTERS.index("trades_dropped")] > 0).all()


def test_chunked_calls_with_append_equal_one_call(eng):
    """The plain form (one call per 100-message chunk, trades appended) gives
    exactly the single-call result."""
    n, per = 12, 2500
    msgs, off = lobgen.generate(lobgen.make_params(77, "three"), [per] * n)
    e = eng.Engine(n, 100, 4096, append_trades=True)
    d = eng.messages_to_device(msgs)
    for c0 in range(0, per, 100):
        c1 = min(per, c0 + 100)
        for b in range(n):
            seg = torch.tensor([b * per + c0, b * per + c1], dtype=torch.int64, device="cuda")
            ids = torch.tensor([b], dtype=torch.int32, device="cuda")
            e.process_batch(d, seg, ids)
    g = gpu_outputs(e)
    ref = oracle.Oracle(n, 100, 4096)
    ref.process(msgs, off)
    assert_same(g, oracle_outputs(ref))


def test_chunk_major_layout_plain_form(eng):
    """Messages laid out chunk-major ([chunk][book][100]) and processed with one
    launch per chunk, trades appended: identical to one call per book stream."""
    n, per, ch = 16, 1000, 100
    msgs, off = lobgen.generate(lobgen.make_params(78, "three"), [per] * n)
    cm = np.ascontiguousarray(msgs.reshape(n, per // ch, ch).transpose(1, 0, 2)).reshape(-1)
    e = eng.Engine(n, 100, 4096, append_trades=True)
    d = eng.messages_to_device(cm)
    for c in range(per // ch):
        seg = torch.arange(0, n * ch + 1, ch, dtype=torch.int64, device="cuda") + c * n * ch
        e.process_batch(d, seg)
    ref = oracle.Oracle(n, 100, 4096)
    ref.process(msgs, off)
    assert_same(gpu_outputs(e), oracle_outputs(ref))


def test_book_subsets_and_empty_segments(eng):
    n = 40
    p = lobgen.make_params(9)
    hs = lobgen.HostStreams(p, n)
    e = eng.Engine(n, 100, 2048)
    ref = oracle.Oracle(n, 100, 2048)
    rng = np.random.default_rng(3)
    for step in range(6):
        ids = np.sort(rng.choice(n, size=int(rng.integers(1, n + 1)), replace=False)).astype(np.int32)
        counts = np.zeros(n, np.int64)
        counts[ids] = rng.integers(0, 400, size=len(ids))
        all_m, all_off = hs.advance(counts)
        seg_counts = counts[ids]
        seg_m = np.concatenate([all_m[all_off[b]:all_off[b + 1]] for b in ids])
        seg_off = lobgen.offsets_from_counts(seg_counts)
        e.process_batch(eng.messages_to_device(seg_m) if len(seg_m) else
                        torch.zeros((1, 8), dtype=torch.int32, device="cuda"),
                        torch.from_numpy(seg_off).cuda(), torch.from_numpy(ids).cuda())
        ref.process(seg_m, seg_off, ids)
        assert_same(gpu_outputs(e), oracle_outputs(ref))


def test_set_book_roundtrip_and_continue(eng):
    hs = lobgen.HostStreams(lobgen.make_params(21), 8)
    msgs, off = hs.advance([3000] * 8)
    ref = oracle.Oracle(8, 100, 4096)
    ref.process(msgs, off)
    bk = ref.book()
    e = eng.Engine(8, 100, 4096)
    e.set_book({k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in bk.items()})
    g = e.book()
    for k, v in bk.items():
        assert np.array_equal(g[k].cpu().numpy(), v)
    more, moff = hs.advance([1500] * 8)
    e.process_batch(eng.messages_to_device(more), torch.from_numpy(moff).cuda())
    ref2 = oracle.Oracle(8, 100, 4096)
    ref2.set_book(bk)
    ref2.process(more, moff)
    got = gpu_outputs(e)
    exp = oracle_outputs(ref2)
    for k in exp:
        if k != "counters":
            assert_same({k: got[k]}, {k: exp[k]})


def test_bad_book_load_sets_status(eng):
    e = eng.Engine(2, 8, 16)
    shp = (2, 2, 8)
    px = torch.full(shp, -1, dtype=torch.int32, device="cuda")
    px[0, 0, :3] = torch.tensor([100, 101, 99], dtype=torch.int32)  # bids not descending
    qty = torch.ones(shp, dtype=torch.int32, device="cuda")
    cnt = torch.zeros((2, 2), dtype=torch.int32, device="cuda")
    cnt[0, 0] = 3
    e.set_book(dict(price=px, qty=qty, oid=qty.clone(), tid=qty.clone(),
                    time_ns=torch.ones(shp, dtype=torch.int64, device="cuda"), count=cnt))
    _, st = e.stats()
    assert int(st.item()) & eng.STATUS_BAD_BOOK_LOAD
    assert int(e.book()["count"][0, 0].item()) == 0


def test_out_of_range_book_id_is_skipped_and_flagged(eng):
    msgs, off = lobgen.generate(lobgen.make_params(1), [50, 50])
    e = eng.Engine(4, 100, 64)
    ids = torch.tensor([1, 7], dtype=torch.int32, device="cuda")
    e.process_batch(eng.messages_to_device(msgs), torch.from_numpy(off).cuda(), ids)
    ctr, st = e.stats()
    assert int(st.item()) & eng.STATUS_BAD_BOOK
    c = ctr.cpu().numpy()
    assert c[1, 0] == 50 and c[[0, 2, 3], 0].sum() == 0


def test_argument_errors(eng):
    e = eng.Engine(4, 100, 64)
    with pytest.raises(eng.LobError):
        e.set_launch(0, 64)
    with pytest.raises(eng.LobError):
        e.set_launch(4, 12)
    with pytest.raises(eng.LobError):
        e.levels(65)
    m = torch.zeros((9, 8), dtype=torch.int32, device="cuda")
    off = torch.tensor([0, 1, 2], dtype=torch.int64, device="cuda")
    with pytest.raises(eng.LobError):  # no book ids and n_active != n_books
        e.process_batch(m, off)
    with pytest.raises(eng.LobError):  # misaligned messages
        eng.lob_process_batch(e.h, m.view(-1)[1:], off, torch.tensor([0, 1], dtype=torch.int32,
                                                                      device="cuda"))
    with pytest.raises(eng.LobError):
        eng.Engine(1, 513, 8)
    with pytest.raises(eng.LobError):
        eng.Engine(0, 100, 8)


def test_contexts_with_different_launch_shapes_coexist(eng):
    """Configuring one context (smaller shape) never invalidates another's."""
    msgs, off = lobgen.generate(lobgen.make_params(8), [3000] * 16)
    d, o = eng.messages_to_device(msgs), torch.from_numpy(off).cuda()
    big = eng.Engine(16, 100, 4096)
    big.set_launch(8, 256, 0)
    small = eng.Engine(16, 100, 4096)
    small.set_launch(1, 8, 0)
    big.process_batch(d, o)
    small.process_batch(d, o)
    assert_same(gpu_outputs(big), gpu_outputs(small))


@pytest.mark.parametrize("cap", [7, 100, 250, 500])
def test_level1_trace_matches_oracle(eng, cap):
    counts = [2500, 0, 1, 1999, 4096, 300]
    msgs, off = lobgen.generate(lobgen.make_params(4000 + cap), counts)
    e = eng.Engine(len(counts), cap, 4096)
    l1 = torch.full((len(msgs), 4), -7, dtype=torch.int32, device="cuda")
    eng.lob_process_batch_l1(e.h, eng.messages_to_device(msgs), torch.from_numpy(off).cuda(), l1)
    o = oracle.Oracle(len(counts), cap, 4096)
    exp = o.process_l1(msgs, off)
    assert np.array_equal(l1.cpu().numpy(), exp)
    # the traced run leaves the same books and trades as an untraced one
    assert_same(gpu_outputs(e), oracle_outputs(o))


@pytest.mark.parametrize("chunk", [777, 5000, 12000])
def test_process_host_equals_device_batch(eng, chunk):
    # host-streamed ingest (copy of chunk k overlapping the processing of
    # chunk k-1) gives exactly the one-call result, ragged last chunk included
    n, per, cap, tcap = 64, 5000, 100, 5000
    msgs, off = lobgen.generate(lobgen.make_params(4321, "pm1"), [per] * n)
    ref = eng.Engine(n, cap, tcap)
    ref.process_batch(eng.messages_to_device(msgs), torch.from_numpy(off).cuda())
    want = gpu_outputs(ref)
    ref.close()
    h = torch.from_numpy(msgs.view(np.int32).reshape(-1, 8)).pin_memory()
    e = eng.Engine(n, cap, tcap)
    for _ in range(2):  # the second call reuses the staging buffers
        e.reset()
        e.process_host(h, per, chunk)
        assert_same(gpu_outputs(e), want)
    e.process_host(h[: n * 0], 0, chunk)  # nothing to do
    e.reset()
    e.process_host(h, per, 2 * chunk)  # a larger chunk regrows the staging
    assert_same(gpu_outputs(e), want)
    e.close()


def test_clear_trades_and_reset_books_mid_stream(eng):
    # two halves of every book's stream with appended trade logs; between them
    # the logs are cleared and a subset of books is emptied (a serving slot
    # handed to a new episode): those restart from empty on the second half
    n, per, cap, tcap = 12, 3000, 100, 4000
    msgs, off = lobgen.generate(lobgen.make_params(8080, "pm1"), [per] * n)
    half = per // 2
    first = np.concatenate([msgs[off[b]:off[b] + half] for b in range(n)])
    second = np.concatenate([msgs[off[b] + half:off[b + 1]] for b in range(n)])
    o1 = np.arange(0, n * half + 1, half, dtype=np.int64)
    o2 = np.arange(0, n * (per - half) + 1, per - half, dtype=np.int64)
    reset = np.array([1, 4, 5, 11], np.int32)
    keep = np.setdiff1d(np.arange(n), reset)

    e = eng.Engine(n, cap, tcap, append_trades=True)
    launches0 = eng.lob_launch_count(e.h)
    e.process_batch(eng.messages_to_device(first), torch.from_numpy(o1).cuda())
    e.clear_trades()
    e.reset_books(torch.from_numpy(reset).cuda())
    e.process_batch(eng.messages_to_device(second), torch.from_numpy(o2).cuda())
    g = gpu_outputs(e)
    assert eng.lob_launch_count(e.h) >= launches0 + 2
    e.close()

    # kept books: both halves, logs cleared in between; counters of both halves
    ok = oracle.Oracle(n, cap, tcap, append_trades=True)
    ok.process(first, o1)
    ok.clear_trades()
    ok.process(second, o2)
    rk = oracle_outputs(ok)
    # reset books: the second half alone, from empty, with fresh counters
    orr = oracle.Oracle(n, cap, tcap, append_trades=True)
    orr.process(second, o2)
    rr = oracle_outputs(orr)
    for key in rk:
        if key == "status":
            assert g["status"] == 0
            continue
        assert np.array_equal(g[key][keep], rk[key][keep]), key
        assert np.array_equal(g[key][reset], rr[key][reset]), key
