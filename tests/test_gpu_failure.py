"""Failure handling on the GPU without faulting it.

Every staged copy in the processing and environment kernels is awaited with
a bounded wait (an mbarrier polled against %globaltimer); when it runs out
the warp records LOB_STATUS_TIMEOUT and leaves instead of hanging.  The
self-test entry point runs that same wait on an mbarrier that nothing
completes, with a short limit, so the timeout path is exercised for real;
the device must stay usable afterwards.  Device-side anomalies that need no
timeout (bad book ids, bad segments, bad book loads) are covered by the
parity tests.
"""
import numpy as np
import pytest
import torch

import lobgen
from engine_harness import run_both, assert_same

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    import paper_2308_13289_b300 as eng
    from paper_2308_13289_b300 import build
    build.build()
    return eng


def test_bounded_wait_times_out_and_reports(eng):
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    elapsed = torch.zeros(1, dtype=torch.int64, device="cuda")
    limit_ns = 50_000_000  # 50 ms
    eng.lob_selftest_wait(limit_ns, status, elapsed)
    torch.cuda.synchronize()
    assert int(status.item()) & eng.STATUS_TIMEOUT
    waited = int(elapsed.item())
    assert limit_ns <= waited < 1_000_000_000, waited


def test_device_usable_after_timeout(eng):
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    eng.lob_selftest_wait(10_000_000, status)
    torch.cuda.synchronize()
    assert int(status.item()) & eng.STATUS_TIMEOUT
    msgs, off = lobgen.generate(lobgen.make_params(31), [800] * 8)
    g, r = run_both(msgs, off, 50, 800)
    assert_same(g, r)


def test_selftest_argument_errors(eng):
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(eng.LobError):
        eng.lob_selftest_wait(0, status)
    with pytest.raises(eng.LobError):
        eng.lob_selftest_wait(2_000_000_000, status)
