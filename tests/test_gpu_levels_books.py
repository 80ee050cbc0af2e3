"""lob_get_levels_books: the top levels of the listed books only.

On seeded streams at a register-resident and a shared-memory capacity, the
rows of the listed books equal what lob_get_levels writes for every book (and
the oracle's levels), the other rows keep what the caller put there, an id
outside the batch sets LOB_STATUS_BAD_BOOK without stopping the rest, and an
empty list writes nothing.
"""
import numpy as np
import pytest
import torch

import lobgen
import oracle
from engine_harness import oracle_outputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cap", [100, 250])
def test_listed_rows_equal_full_levels_and_oracle(cap):
    import paper_2308_13289_b300 as eng
    n, per, depth = 40, 3000, 10
    m, off = lobgen.generate(lobgen.make_params(77), [per] * n)
    e = eng.Engine(n, cap, per)
    e.process_batch(eng.messages_to_device(m), torch.from_numpy(off).cuda())
    full = [x.cpu().numpy() for x in e.levels(depth)]
    ids = np.array([3, 0, 39, 17, 18, 5], dtype=np.int32)
    got = [x.cpu().numpy() for x in e.levels_of(torch.from_numpy(ids).cuda(), depth)]
    o = oracle.Oracle(n, cap, per, 0)
    o.process(m, off)
    ref = oracle_outputs(o, depth)
    others = np.setdiff1d(np.arange(n), ids)
    for g, f, name in zip(got, full, ("bid_px", "bid_qty", "ask_px", "ask_qty")):
        assert np.array_equal(g[ids], f[ids]), name
        assert np.array_equal(g[ids], ref[name][ids]), name
        assert (g[others] == -7).all(), name
    _, st = e.stats()
    assert int(st.item()) == 0
    e.close()


def test_bad_id_is_flagged_and_skipped_and_empty_list_writes_nothing():
    import paper_2308_13289_b300 as eng
    n, depth = 8, 5
    m, off = lobgen.generate(lobgen.make_params(78), [500] * n)
    e = eng.Engine(n, 100, 500)
    e.process_batch(eng.messages_to_device(m), torch.from_numpy(off).cuda())
    full = [x.cpu().numpy() for x in e.levels(depth)]
    ids = torch.tensor([2, n, 6, -1], dtype=torch.int32, device="cuda")
    got = [x.cpu().numpy() for x in e.levels_of(ids, depth)]
    for g, f in zip(got, full):
        assert np.array_equal(g[[2, 6]], f[[2, 6]])
        assert (g[[0, 1, 3, 4, 5, 7]] == -7).all()
    _, st = e.stats()
    assert int(st.item()) & eng.STATUS_BAD_BOOK
    e.close()
    e2 = eng.Engine(n, 100, 500)
    got = [x.cpu().numpy() for x in e2.levels_of(torch.empty(0, dtype=torch.int32,
                                                             device="cuda"), depth)]
    torch.cuda.synchronize()
    assert all((g == -7).all() for g in got)
    e2.close()
