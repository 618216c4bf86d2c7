"""Host logic of batched solves: the largest-first (LPT) scheduler behind
dgamp_ct_solve_batched and the split of a batch across processes.  Runs the
library's host-only entry point; no device work."""
import itertools

import numpy as np
import pytest

import synth

dg = pytest.importorskip("paper_1609_04661_gb300")


@pytest.fixture(scope="module")
def lib():
    from paper_1609_04661_gb300 import build
    build.build()
    return dg.load()


def brute_makespan(work, m):
    best = None
    for assign in itertools.product(range(m), repeat=len(work)):
        loads = np.zeros(m, dtype=np.int64)
        for w, q in zip(work, assign):
            loads[q] += w
        best = loads.max() if best is None else min(best, loads.max())
    return best


def test_hand_example(lib):
    # largest first: 7 -> q0, 5 -> q1, 4 -> q1 (5 < 7), 3 -> q0 (7 < 9), 1 -> q1 (9 < 10)
    q, load = dg.schedule_lpt([3, 7, 1, 5, 4], 2)
    assert list(q) == [0, 0, 1, 1, 1]
    assert list(load) == [10, 10]


def test_ties_keep_input_order_and_lowest_queue(lib):
    q, load = dg.schedule_lpt([5, 5, 5, 5], 3)
    assert list(q) == [0, 1, 2, 0]
    assert list(load) == [10, 5, 5]


def test_lpt_is_within_grahams_bound_of_the_optimum(lib):
    """Graham (1969): LPT's makespan is at most (4/3 - 1/(3m)) times the optimum."""
    rng = np.random.default_rng(4)
    for trial in range(40):
        m = int(rng.integers(2, 4))
        work = rng.integers(1, 50, size=int(rng.integers(3, 8)))
        q, load = dg.schedule_lpt(work, m)
        assert load.sum() == work.sum()
        assert all(load[k] == work[q == k].sum() for k in range(m))
        opt = brute_makespan(list(work), m)
        assert load.max() <= (4.0 / 3.0 - 1.0 / (3 * m)) * opt + 1e-9


def test_more_queues_than_jobs_and_empty(lib):
    q, load = dg.schedule_lpt([4, 9], 5)
    assert list(q) == [1, 0] and list(load) == [9, 4, 0, 0, 0]
    q, load = dg.schedule_lpt([], 3)
    assert q.size == 0 and list(load) == [0, 0, 0]


def test_bad_arguments_are_rejected(lib):
    with pytest.raises(dg.DgampError):
        dg.schedule_lpt([1, -2], 2)
    with pytest.raises(dg.DgampError):
        dg.schedule_lpt([1, 2], 0)


def test_mixed_batch_split_across_ranks_is_balanced(lib):
    """The 64-slice mixed batch split over 2, 4 and 8 processes: every slice
    placed once, and no rank above the LPT bound of the mean load."""
    batch = synth.make_batch("mixed64")
    work = np.array([c["n_views"] * c["n_det"] * c["n"] for c in batch], dtype=np.int64)
    for ranks in (2, 4, 8):
        q, load = dg.schedule_lpt(work, ranks)
        assert np.bincount(q, minlength=ranks).sum() == work.size and load.sum() == work.sum()
        # a lower bound on the optimum is max(mean load, largest job)
        lb = max(work.sum() / ranks, work.max())
        assert load.max() <= (4.0 / 3.0) * lb
