"""The device generator draws exactly the host generator's streams."""
import numpy as np
import pytest
import torch

import lobgen

pytestmark = pytest.mark.gpu


def test_device_streams_equal_host_streams():
    lobgen.build(cuda=True)
    for walk, pool in (("pm1", 64), ("three", 7), ("pm1", 4096)):
        p = lobgen.make_params(2468, walk, pool_cap=pool)
        counts = [3000, 1, 0, 4500, 777] * 10
        host, hoff = lobgen.generate(p, counts)
        ds = lobgen.DeviceStreams(p, len(counts))
        dev, doff = ds.advance(counts)
        assert np.array_equal(doff.cpu().numpy(), hoff)
        assert np.array_equal(dev.cpu().numpy(), host.view(np.int32).reshape(-1, 8))


def test_device_streams_resume_and_select_books():
    p = lobgen.make_params(1357)
    hs = lobgen.HostStreams(p, 20)
    ds = lobgen.DeviceStreams(p, 20)
    for step in range(3):
        ids = np.arange(step, 20, 3, dtype=np.int32)
        counts = np.zeros(20, np.int64)
        counts[ids] = 100 + step
        hm, hoff = hs.advance(counts)
        dm, doff = ds.advance(counts[ids], ids=ids)
        exp = np.concatenate([hm[hoff[b]:hoff[b + 1]] for b in ids])
        assert np.array_equal(dm.cpu().numpy(), exp.view(np.int32).reshape(-1, 8))


def test_device_agent_draws_equal_host():
    d = lobgen.agent_draws_device(99, 300, 17, step0=5).cpu().numpy().view(np.uint32)
    h = lobgen.agent_draws(99, 300, 22)[5:]
    assert np.array_equal(d, h)
