"""Oracle of the split expansion's merge schedule (Section IV, "Binary
merge"; Algorithm 2) and of the memory it holds.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``; the product path never
imports it, and nothing here imports the product path.

The expansion B = A A is split along its inner index k into ``nstages``
blocks K_t = [(t-1) n / nstages, t n / nstages); stage t forms the partial
product P_t = A(:, K_t) A(K_t, :).  Algorithm 2 keeps the partial products
on a stack: after stage t is pushed, the top nmerges + 1 lists are merged
into one, nmerges being the number of times t halves evenly (0 for odd t).
Lists left on the stack after the last stage are merged together.  A
multiway merge instead holds every P_t at once (Section IV compares the two
in memory).

Only patterns matter for the memory: the entries of A are positive, so the
pattern of a sum of partial products is the union of their patterns.  The
patterns come from a sparse product of 0/1 matrices (a library matmul as one
step: entry (i, j) counts the paths i <- k <- j, never zero where a path
exists).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp


@dataclasses.dataclass
class MergeStats:
    stages: int
    merges: int
    partial_entries: int        # sum_t nnz(P_t): what a multiway merge holds
    binary_peak_entries: int    # the largest merge's input entries
    live_peak_entries: int      # most entries held at once (stack + a merge's output)
    merged_entries: int         # nnz(A A)


def stage_blocks(n: int, nstages: int):
    """The blocks K_t of the inner index, t = 1 .. nstages."""
    return [((t - 1) * n // nstages, t * n // nstages) for t in range(1, nstages + 1)]


def _pattern(A):
    """0/1 CSC matrix with the pattern of A (A: an object with n, colptr, rowidx)."""
    n = int(A.n)
    nnz = int(A.colptr[n]) if n else 0
    return sp.csc_matrix((np.ones(nnz), np.asarray(A.rowidx[:nnz]), np.asarray(A.colptr)),
                         shape=(n, n))


def partial_patterns(A, nstages: int):
    """Patterns of P_t = A(:, K_t) A(K_t, :) for every stage t."""
    M = _pattern(A)
    out = []
    for k0, k1 in stage_blocks(int(A.n), nstages):
        P = (M[:, k0:k1] @ M[k0:k1, :]).tocsc()
        P.data[:] = 1.0
        out.append(P)
    return out


def trailing_halvings(t: int) -> int:
    """nmerges of Algorithm 2 for stage t: how many times t divides by 2."""
    m = 0
    while t > 0 and t % 2 == 0:
        t //= 2
        m += 1
    return m


def binary_merge(A, nstages: int) -> MergeStats:
    """Run Algorithm 2's schedule over the partial patterns and record its memory."""
    parts = partial_patterns(A, nstages)
    stack = []
    live = 0
    st = MergeStats(stages=nstages, merges=0, partial_entries=0, binary_peak_entries=0,
                    live_peak_entries=0, merged_entries=0)

    def merge(count):
        nonlocal live
        top = stack[-count:]
        inputs = sum(P.nnz for P in top)
        M = top[0]
        for P in top[1:]:
            M = M + P
        M = M.tocsc()
        M.data[:] = 1.0
        st.binary_peak_entries = max(st.binary_peak_entries, inputs)
        live += M.nnz
        st.live_peak_entries = max(st.live_peak_entries, live)
        del stack[-count:]
        live -= inputs
        stack.append(M)
        st.merges += 1

    for t, P in enumerate(parts, start=1):
        st.partial_entries += P.nnz
        stack.append(P)
        live += P.nnz
        st.live_peak_entries = max(st.live_peak_entries, live)
        nm = trailing_halvings(t)
        if nm > 0:
            merge(min(nm + 1, len(stack)))
    if len(stack) > 1:
        merge(len(stack))
    st.merged_entries = stack[-1].nnz if stack else 0
    return st
