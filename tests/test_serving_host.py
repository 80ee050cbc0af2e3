"""Host-side logic of the serving loop (no GPU): the HBM footprint an episode
is admitted by, and the seeded arrival process."""
import numpy as np

from paper_2308_13289_b300 import serve


def test_footprint_counts_book_log_generator_and_window():
    # book state of 128 (cap 100), 32 (cap 7) and 512 (cap 500) slots at 48 B
    assert serve.book_bytes(100) == 6144
    assert serve.book_bytes(7) == 1536
    assert serve.book_bytes(500) == 24576
    # generator state: 40 B of stream state + 64 remembered ids of 16 B
    assert serve.GEN_STATE_BYTES == 40 + 64 * 16
    base = serve.footprint_bytes(100, 0, 0)
    assert base == 6144 + 8 + 8 + 8 * 20 + 40 + 64 * 16
    # the trade log and the step window (32 B per message) are counted
    assert serve.footprint_bytes(100, 2048, 0) - base == 32 * 2048
    assert serve.footprint_bytes(100, 0, 500) - base == 32 * 500


def test_poisson_arrivals_match_the_workload():
    eps = serve.sample_episodes(2000.0, 2.0, 7)
    t = np.array([e.arrival for e in eps])
    assert (np.diff(t) > 0).all() and t[-1] < 2.0
    assert 3800 < len(eps) < 4200  # 2,000/s over 2 s
    caps = np.array([e.capacity for e in eps])
    assert set(caps) == {100, 250, 500}
    steps = np.array([e.n_steps for e in eps])
    mps = np.array([e.msgs_per_step for e in eps])
    assert steps.min() >= 200 and steps.max() <= 2000
    assert mps.min() >= 100 and mps.max() <= 500
    # the same seed gives the same requests
    again = serve.sample_episodes(2000.0, 2.0, 7)
    assert [(e.capacity, e.n_steps, e.msgs_per_step) for e in again] == \
        [(e.capacity, e.n_steps, e.msgs_per_step) for e in eps]
