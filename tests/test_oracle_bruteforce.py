"""Brute force on tiny books: every message sequence over a small alphabet is
run through the ordered-map oracle and through the paper-literal unsorted-array
implementation (Sec. 4 eqs. 1-2, Sec. 4.1); books, trades and counters must be
identical.  The two share no code, so a dropped term, a wrong sign or a wrong
index in either shows up as a mismatch."""
import itertools

import numpy as np
import pytest

import oracle


def _alphabet():
    """Per-position choices: limit (S, P, Q), market (S, Q), cancel/delete of
    the id issued 1 or 2 messages earlier (its own side or the other side)."""
    out = []
    for s in (1, -1):
        for p in (1, 2, 3):
            for q in (1, 2):
                out.append(("L", s, p, q))
    for s in (1, -1):
        for q in (1, 3):
            out.append(("M", s, 0, q))
    for t in (2, 3):
        for back in (1, 2):
            for q in (1, 2):
                out.append(("C", t, back, q))
    out.append(("C", 2, 1, 9))  # cancel larger than any order
    out.append(("W", 2, 1, 1))  # cancel naming the other side
    return out


def _encode(seqs, alphabet):
    rows = []
    for seq in seqs:
        sides = {}
        for i, a in enumerate(seq):
            oid = i + 1
            tm = 100 + i
            kind = alphabet[a]
            if kind[0] == "L":
                _, s, p, q = kind
                rows.append((1, s, p, q, oid, 10 + oid, tm))
                sides[oid] = (s, p)
            elif kind[0] == "M":
                _, s, _, q = kind
                rows.append((4, s, 0, q, oid, 10 + oid, tm))
                sides[oid] = (s, 0)
            else:
                _, t, back, q = kind
                tgt = oid - back
                s, p = sides.get(tgt, (1, 1))
                if kind[0] == "W":
                    s = -s
                rows.append((t, s, p, q, max(tgt, 0), 10 + oid, tm))
    return oracle.messages(rows)


def _compare(seqs, alphabet, cap, rule, L):
    m = _encode(seqs, alphabet)
    n = len(seqs)
    off = np.arange(0, n * L + 1, L, dtype=np.int64)
    o = oracle.Oracle(n, cap, 8, rule)
    o.process(m, off)
    bk, tr, cnt = o.book(), *o.trades()
    lbk, ltr, lcnt, lctr = oracle.literal_run(m, off, cap, 8, rule)
    for k in bk:
        bad = np.nonzero((bk[k] != lbk[k]).reshape(n, -1).any(1))[0]
        assert len(bad) == 0, (k, seqs[bad[0]])
    assert np.array_equal(cnt, lcnt)
    assert np.array_equal(tr.view(np.int32), ltr.view(np.int32))
    assert np.array_equal(o.counters(), lctr)


@pytest.mark.parametrize("cap,rule", [(2, 0), (2, 1), (3, 0)])
def test_exhaustive_length4(cap, rule):
    alphabet = _alphabet()
    seqs = list(itertools.product(range(len(alphabet)), repeat=4))
    _compare(seqs, alphabet, cap, rule, 4)


@pytest.mark.parametrize("cap,rule,seed", [(2, 0, 1), (3, 1, 2), (1, 0, 3), (4, 0, 4)])
def test_random_length8(cap, rule, seed):
    alphabet = _alphabet()
    rng = np.random.default_rng(seed)
    seqs = [tuple(r) for r in rng.integers(0, len(alphabet), size=(60_000, 8))]
    _compare(seqs, alphabet, cap, rule, 8)
