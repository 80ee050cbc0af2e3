"""The allocation-free entry point lob_process_streams_static.

Some callers cannot allocate device memory while they run (a service that
reserved the GPU's memory for its own pool up front, or a latency-critical
loop where cudaMalloc/cudaFree would synchronise the device).  For them the
library offers one call that needs no context and keeps its scratch in a fixed
array inside the library.  This file checks, through the C ABI, that two calls
in a row give exactly (bit for bit, the tolerance of every engine test) what
the context-based entry points give on the same inputs, and that a request
larger than the fixed scratch is refused.  It is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

import lobgen

pytestmark = pytest.mark.gpu


def _lib():
    from paper_2308_13289_b300 import build
    lib = ctypes.CDLL(build.build())
    vp, i32 = ctypes.c_void_p, ctypes.c_int32
    lib.lob_process_streams_static.restype = ctypes.c_int
    lib.lob_process_streams_static.argtypes = [vp, vp, i32, i32, i32, i32] + [vp] * 11
    lib.lob_last_error.restype = ctypes.c_char_p
    return lib


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _static_call(lib, msgs, off, n, cap, tcap, rule):
    dev = "cuda"
    out = dict(
        trades=torch.full((n, tcap, 8), -1, dtype=torch.int32, device=dev),
        trade_counts=torch.empty(n, dtype=torch.int64, device=dev),
        counters=torch.full((n, 20), 123, dtype=torch.int64, device=dev),
        price=torch.empty((n, 2, cap), dtype=torch.int32, device=dev),
        qty=torch.empty((n, 2, cap), dtype=torch.int32, device=dev),
        oid=torch.empty((n, 2, cap), dtype=torch.int32, device=dev),
        tid=torch.empty((n, 2, cap), dtype=torch.int32, device=dev),
        time_ns=torch.empty((n, 2, cap), dtype=torch.int64, device=dev),
        count=torch.empty((n, 2), dtype=torch.int32, device=dev),
        status=torch.full((1,), 77, dtype=torch.int32, device=dev))
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.lob_process_streams_static(
        _p(msgs), _p(off), n, cap, tcap, rule, _p(out["trades"]), _p(out["trade_counts"]),
        _p(out["counters"]), _p(out["price"]), _p(out["qty"]), _p(out["oid"]), _p(out["tid"]),
        _p(out["time_ns"]), _p(out["count"]), _p(out["status"]), stream)
    assert rc == 0, lib.lob_last_error()
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _context_call(msgs, off, n, cap, tcap, rule):
    import paper_2308_13289_b300 as eng
    e = eng.Engine(n, cap, tcap, rule)
    e.process_batch(msgs, off)
    bk = e.book()
    tr, cnt = e.trades()
    ctr, st = e.stats()
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy() for k, v in bk.items()}
    out.update(trades=tr.cpu().numpy(), trade_counts=cnt.cpu().numpy(),
               counters=ctr.cpu().numpy(), status=st.cpu().numpy())
    e.close()
    return out


def test_static_entry_point_matches_context_entry_points_twice():
    import paper_2308_13289_b300 as eng
    lib = _lib()
    # two different calls in a row; the second is smaller, so stale contents
    # of the shared scratch from the first would show up as differences
    for seed, n, per, cap, rule in ((314, 24, 3000, 100, 0), (2718, 9, 2000, 250, 1)):
        m, off = lobgen.generate(lobgen.make_params(seed), [per] * n)
        dm = eng.messages_to_device(m)
        doff = torch.from_numpy(off).cuda()
        tcap = per
        got = _static_call(lib, dm, doff, n, cap, tcap, rule)
        exp = _context_call(dm, doff, n, cap, tcap, rule)
        for k in exp:
            assert np.array_equal(got[k], exp[k]), (seed, k)
        assert int(got["status"][0]) == 0


def test_static_entry_point_refuses_oversized_requests():
    lib = _lib()
    m = torch.zeros((8, 8), dtype=torch.int32, device="cuda")
    off = torch.zeros(100_001, dtype=torch.int64, device="cuda")
    cnt = torch.zeros(100_000, dtype=torch.int64, device="cuda")
    rc = lib.lob_process_streams_static(_p(m), _p(off), 100_000, 100, 0, 0, None, _p(cnt),
                                        _p(cnt), None, None, None, None, None, None, _p(m),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == -1
    assert b"scratch" in lib.lob_last_error()


@pytest.mark.parametrize("cap,n_max", [(100, 5454), (512, 1364)])
def test_static_entry_point_size_limit_is_exact(cap, n_max):
    """256 + roundup(8 n, 256) + n * 48 * S <= 32 MiB (S = capacity rounded up
    to 128 or 512 slots here): the largest n is accepted, n + 1 is refused.
    Every segment is empty, so the accepted call only clears its outputs."""
    lib = _lib()
    m = torch.zeros((8, 8), dtype=torch.int32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for n, rc_want in ((n_max, 0), (n_max + 1, -1)):
        off = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
        cnt = torch.full((n,), 9, dtype=torch.int64, device="cuda")
        ctr = torch.full((n, 20), 9, dtype=torch.int64, device="cuda")
        st = torch.full((1,), 9, dtype=torch.int32, device="cuda")
        rc = lib.lob_process_streams_static(_p(m), _p(off), n, cap, 0, 0, None, _p(cnt), _p(ctr),
                                            None, None, None, None, None, None, _p(st), stream)
        assert rc == rc_want, (n, lib.lob_last_error())
        if rc == 0:
            torch.cuda.synchronize()
            assert int(cnt.abs().sum()) == 0 and int(ctr.abs().sum()) == 0 and int(st.item()) == 0
        else:
            assert ("at most %d books" % n_max).encode() in lib.lob_last_error()
