"""The seeded input generator: determinism, the stated recipe, and exactness
of its integer-only sampling tables."""
from fractions import Fraction

import numpy as np

import lobgen


def test_geometric_thresholds_are_exact():
    # thr[k] = floor(2^64 * (1 - (1-p)^(k+1))) checked with exact fractions
    for p, tab in ((Fraction(3, 10), lobgen.GEO_PX), (Fraction(2, 100), lobgen.GEO_Q)):
        for k in (0, 1, 2, 7, 30, len(tab) - 1):
            exact = (1 << 64) * (1 - (1 - p) ** (k + 1))
            v = min(int(exact), (1 << 64) - 1)  # floor for positive values
            assert int(tab[k]) == v
        assert (np.diff(tab.astype(object)) >= 0).all()
    # first thresholds: P(G=0) = p
    assert int(lobgen.GEO_PX[0]) == int(Fraction(3, 10) * (1 << 64))


def test_streams_are_deterministic_and_thread_independent():
    p = lobgen.make_params(123)
    a, oa = lobgen.generate(p, [5000] * 8, threads=1)
    b, ob = lobgen.generate(p, [5000] * 8, threads=8)
    assert np.array_equal(a, b) and np.array_equal(oa, ob)
    c, _ = lobgen.generate(lobgen.make_params(124), [5000] * 8)
    assert not np.array_equal(a, c)


def test_resumable_streams_equal_one_shot():
    p = lobgen.make_params(77, "three")
    whole, _ = lobgen.generate(p, [3000] * 4)
    hs = lobgen.HostStreams(p, 4)
    parts = [hs.advance([1000] * 4)[0].reshape(4, 1000) for _ in range(3)]
    joined = np.concatenate(parts, axis=1).reshape(-1)
    assert np.array_equal(joined, whole)


def test_recipe_statistics():
    p = lobgen.make_params(20230825)
    m, off = lobgen.generate(p, [50_000] * 8)
    frac = np.bincount(m["type"], minlength=5)[1:] / len(m)
    # cancels/deletes drawn while the id pool is empty become adds (rare)
    assert abs(frac[0] - 0.55) < 0.01 and abs(frac[1] - 0.25) < 0.01
    assert abs(frac[2] - 0.12) < 0.01 and abs(frac[3] - 0.08) < 0.01
    assert abs((m["side"] == 1).mean() - 0.5) < 0.01
    mk = m[m["type"] == 4]
    assert (mk["price"] == 0).all()
    q = mk["qty"].astype(np.float64)
    assert abs(q.mean() - 50.0) < 1.5  # 1 + geometric(0.02): mean 1 + 0.98/0.02
    tid = m["tid"]
    assert tid.min() >= 1 and tid.max() <= 1000
    for b in range(8):
        s = m[off[b]:off[b + 1]]
        dt = np.diff(s["time_ns"])
        assert dt.min() >= 1 and dt.max() <= 1000
        new = s[(s["type"] == 1) | (s["type"] == 4)]
        assert (np.diff(new["oid"]) == 1).all() and new["oid"][0] == 1


def test_cancels_target_earlier_limit_orders():
    p = lobgen.make_params(5)
    m, _ = lobgen.generate(p, [20_000])
    orig = {}
    for r in m:
        if r["type"] == 1:
            orig[int(r["oid"])] = (int(r["side"]), int(r["price"]), int(r["qty"]))
        elif r["type"] in (2, 3):
            s, px, q = orig[int(r["oid"])]
            assert (int(r["side"]), int(r["price"])) == (s, px)
            if r["type"] == 3:
                assert int(r["qty"]) == q
            else:
                assert 1 <= int(r["qty"]) <= max(1, q - 1)


def test_price_offsets_follow_the_recipe():
    p = lobgen.make_params(9, "none")  # frozen mid = 10,000
    m, _ = lobgen.generate(p, [40_000])
    lim = m[m["type"] == 1]
    # passive buys at mid-1-G (< mid), aggressive buys at mid+G (>= mid)
    buys = lim[lim["side"] == 1]["price"] - 10_000
    sells = 10_000 - lim[lim["side"] == -1]["price"]
    for d in (buys, sells):
        aggressive = (d >= 0).mean()
        assert abs(aggressive - 0.10) < 0.01
        passive = -d[d < 0] - 1  # G
        assert abs((passive == 0).mean() - 0.3) < 0.02


def test_agent_draws_are_uniform():
    d = lobgen.agent_draws(1, 4096, 50)
    n = (d & 3) + 1
    assert n.min() == 1 and n.max() == 4
    acts = np.stack([(d >> (2 + 3 * k)) & 7 for k in range(4)])
    assert acts.max() == 5
    freq = np.bincount(acts.reshape(-1), minlength=6) / acts.size
    assert np.abs(freq - 1 / 6).max() < 0.01
