"""Multi-rank host logic: books shard across ranks with no data-path
collective (books are independent, Sec. 4.3); only timing is combined."""
from __future__ import annotations

import os

import numpy as np


def rank_world():
    """(rank, world size, local rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def stream_ids(rank: int, n_per_rank: int) -> np.ndarray:
    """Weak scaling: rank r runs books [r*n, (r+1)*n) of one global id space, so
    every rank's streams are distinct and reproducible."""
    return np.arange(rank * n_per_rank, (rank + 1) * n_per_rank, dtype=np.uint64)


def balanced_ranges(counts, world: int):
    """Strong scaling of uneven books: contiguous book ranges with roughly equal
    message totals; returns [(lo, hi)] per rank."""
    counts = np.asarray(counts, dtype=np.int64)
    csum = np.concatenate([[0], np.cumsum(counts)])
    total = csum[-1]
    cuts = [0]
    for r in range(1, world):
        cuts.append(int(np.searchsorted(csum, total * r / world)))
    cuts.append(len(counts))
    return [(cuts[r], max(cuts[r], cuts[r + 1])) for r in range(world)]


def max_over_ranks(value: float, device=None) -> float:
    """MAX of a float over all ranks of the default process group (identity
    without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
