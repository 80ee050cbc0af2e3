"""Run the CUDA engine and the CPU oracle on the same inputs and compare
their outputs element by element (books, trades, counters, levels)."""
import numpy as np

import oracle

DEPTH = 10


def gpu_outputs(e, depth=DEPTH):
    import torch
    bk = e.book()
    tr, cnt = e.trades()
    lv = e.levels(depth)
    ctr, st = e.stats()
    torch.cuda.synchronize()
    out = {"book_" + k: v.cpu().numpy() for k, v in bk.items()}
    out["trades"] = tr.cpu().numpy()
    out["trade_counts"] = cnt.cpu().numpy()
    for name, v in zip(("bid_px", "bid_qty", "ask_px", "ask_qty"), lv):
        out[name] = v.cpu().numpy()
    out["counters"] = ctr.cpu().numpy()
    out["status"] = int(st.item())
    return out


def oracle_outputs(o, depth=DEPTH):
    out = {"book_" + k: v for k, v in o.book().items()}
    tr, cnt = o.trades()
    out["trades"] = tr.view(np.int32).reshape(o.n_books, o.trade_capacity, 8)
    out["trade_counts"] = cnt
    for name, v in zip(("bid_px", "bid_qty", "ask_px", "ask_qty"), o.levels(depth)):
        out[name] = v
    out["counters"] = o.counters()
    out["status"] = 0
    return out


def assert_same(gpu, ref, books=None):
    """Bit-exact comparison; `books` restricts to a subset of book indices
    (the GPU side may hold more books than the oracle computed)."""
    for k, v in ref.items():
        g = gpu[k]
        if k != "status" and books is not None:
            g = g[books]
        if k == "status":
            assert g == v, "device status word %d" % g
            continue
        if not np.array_equal(g, v):
            diff = np.argwhere(g != v)
            raise AssertionError("%s differs at %d places, first %s: gpu %s oracle %s"
                                 % (k, len(diff), diff[0], g[tuple(diff[0])], v[tuple(diff[0])]))


def run_both(msgs, off, cap, tcap, rule=0, launch=None, depth=DEPTH):
    import torch

    import paper_2308_13289_b300 as eng
    n = len(off) - 1
    e = eng.Engine(n, cap, tcap, rule)
    if launch:
        e.set_launch(*launch)
    e.process_batch(eng.messages_to_device(msgs), torch.from_numpy(off).cuda())
    g = gpu_outputs(e, depth)
    e.close()
    o = oracle.Oracle(n, cap, tcap, rule)
    o.process(msgs, off)
    return g, oracle_outputs(o, depth)
