"""World-size-2 gloo ranks on the CPU: book sharding and max-over-ranks timing
of the multi-GPU path (no data-path collective exists to test)."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

from paper_2308_13289_b300 import dist as ldist


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, _ = ldist.rank_world()
    ids = ldist.stream_ids(r, 1024)
    t = ldist.max_over_ranks(10.0 + 5.0 * r)
    q.put((r, w, int(ids[0]), int(ids[-1]), t))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_books_and_reduce_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][:4] == (0, 2, 0, 1023) and res[1][:4] == (1, 2, 1024, 2047)
    assert res[0][4] == res[1][4] == 15.0  # MAX over ranks


def test_balanced_ranges_cover_books_once():
    counts = np.random.default_rng(0).integers(1000, 200_000, size=4096)
    for world in (1, 2, 3, 8):
        rg = ldist.balanced_ranges(counts, world)
        assert rg[0][0] == 0 and rg[-1][1] == len(counts)
        assert all(a[1] == b[0] for a, b in zip(rg, rg[1:]))
        tot = [counts[lo:hi].sum() for lo, hi in rg]
        assert max(tot) - min(tot) <= counts.max() + 1


def test_single_process_max_is_identity():
    assert ldist.max_over_ranks(3.5) == 3.5


def _failing_worker(rank, world, port, q):
    # rank 1 fails between steps (before the timing reduction); rank 0 must
    # learn it from the process group's timeout, not hang
    import datetime

    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=5))
    if rank == 1:
        q.put((1, "left"))
        q.close()
        q.join_thread()
        os._exit(3)  # the failing rank leaves with its collective not entered
    try:
        ldist.max_over_ranks(1.0)
        q.put((0, "no error"))
    except Exception as exc:  # a timeout or connection error from gloo
        q.put((0, type(exc).__name__))
    q.close()
    q.join_thread()
    os._exit(0)


def test_rank_failure_surfaces_as_an_error_not_a_hang():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_failing_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
    assert res[1] == "left"
    assert res[0] != "no error", res
    assert procs[0].exitcode == 0 and procs[1].exitcode == 3
