"""Pins of the merge-schedule oracle (Section IV, Algorithm 2) against
closed forms of the schedule and brute-force patterns.

* complete pattern, nstages = 2^m: every partial product is full, so the
  schedule's sizes are multiples of n^2: nstages / 2 merges (one per even
  stage), the last merge pops m + 1 lists, and at most m + 2 full lists are
  held at once (the stack plus the merge's output);
* nstages = 3: stage 2 merges two lists and the leftover pair is merged last;
* diagonal pattern: the partial products are disjoint, so the merged size is
  the sum of theirs;
* random patterns: partial products equal a triple-loop brute force, and the
  merged pattern equals the pattern of the dense product.
"""
import numpy as np
import pytest

pytest.importorskip("scipy")
from oracle import merge  # noqa: E402
from paper_2002_10083_gb300 import synth  # noqa: E402


class _Pat:
    def __init__(self, dense_bool):
        n = dense_bool.shape[0]
        self.n = n
        cols = [np.flatnonzero(dense_bool[:, j]) for j in range(n)]
        self.colptr = np.concatenate([[0], np.cumsum([len(c) for c in cols])]).astype(np.int64)
        self.rowidx = (np.concatenate(cols) if n else np.zeros(0)).astype(np.int32)


@pytest.mark.parametrize("t,m", [(1, 0), (2, 1), (3, 0), (4, 2), (12, 2), (48, 4), (1024, 10)])
def test_trailing_halvings(t, m):
    assert merge.trailing_halvings(t) == m


@pytest.mark.parametrize("m", [1, 2, 3, 4])
def test_complete_pattern_power_of_two(m):
    n = 2 ** m * 3
    A = _Pat(np.ones((n, n), bool))
    st = merge.binary_merge(A, 2 ** m)
    sq = n * n
    assert st.partial_entries == 2 ** m * sq
    assert st.merged_entries == sq
    assert st.merges == 2 ** (m - 1)
    assert st.binary_peak_entries == (m + 1) * sq
    assert st.live_peak_entries == (m + 2) * sq


def test_complete_pattern_three_stages():
    n = 9
    st = merge.binary_merge(_Pat(np.ones((n, n), bool)), 3)
    assert (st.merges, st.binary_peak_entries, st.live_peak_entries) == (2, 2 * n * n, 3 * n * n)


def test_one_stage_merges_nothing():
    n = 7
    st = merge.binary_merge(_Pat(np.ones((n, n), bool)), 1)
    assert (st.merges, st.binary_peak_entries, st.live_peak_entries) == (0, 0, n * n)
    assert st.partial_entries == st.merged_entries == n * n


@pytest.mark.parametrize("ns", [2, 4, 5, 8])
def test_diagonal_pattern_disjoint(ns):
    n = 40
    st = merge.binary_merge(_Pat(np.eye(n, dtype=bool)), ns)
    assert st.partial_entries == st.merged_entries == n
    # every list ends in the final merge of the whole diagonal
    assert st.binary_peak_entries == n
    assert st.live_peak_entries == 2 * n


@pytest.mark.parametrize("seed,ns", [(0, 3), (1, 4), (2, 7)])
def test_random_patterns_brute_force(seed, ns):
    n = 30
    rng = np.random.default_rng(seed)
    D = rng.random((n, n)) < 0.08
    A = _Pat(D)
    parts = merge.partial_patterns(A, ns)
    union = np.zeros((n, n), bool)
    for (k0, k1), P in zip(merge.stage_blocks(n, ns), parts):
        want = np.zeros((n, n), bool)
        for j in range(n):
            for k in range(k0, k1):
                if D[k, j]:
                    for i in range(n):
                        if D[i, k]:
                            want[i, j] = True
        assert np.array_equal(P.toarray() > 0, want)
        union |= want
    st = merge.binary_merge(A, ns)
    assert st.merged_entries == int(((D.astype(int) @ D.astype(int)) > 0).sum())
    assert st.merged_entries == int(union.sum())
    assert st.partial_entries == sum(P.nnz for P in parts)


def test_stage_blocks_cover_the_inner_index():
    for n, ns in [(10, 3), (7, 7), (5, 8), (0, 2)]:
        b = merge.stage_blocks(n, ns)
        assert b[0][0] == 0 and b[-1][1] == n
        assert all(b[i][1] == b[i + 1][0] for i in range(len(b) - 1))


def test_overlapping_partials_binary_merges_fewer_than_multiway():
    """Section IV's memory measure: a multiway merge holds every partial
    entry, the binary merge at most its largest merge's; with overlapping
    patterns the merged lists shrink on the way, so the largest is smaller."""
    A = synth.chung_lu(n=3000, mean=50.0, d_max=500, seed=1)
    for ns in (4, 8, 13, 16):
        st = merge.binary_merge(A, ns)
        assert st.merged_entries < st.binary_peak_entries < st.partial_entries
        # with the merge output counted, the binary schedule still holds less
        assert st.live_peak_entries < st.partial_entries + st.merged_entries
