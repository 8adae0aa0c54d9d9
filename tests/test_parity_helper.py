"""The GPU-vs-oracle comparison helper on hand-made columns (no GPU): an
entry that ties in FP32 with the value at the oracle's cut may be swapped
(the GPU ranks equal FP32 values by row), a swap across clearly different
values may not."""
import numpy as np

import oracle
from paper_2002_10083_gb300 import synth
from tests.parity import compare_iteration


def _column_case(vals):
    """A = unit columns 0..m-1 plus column m holding vals, so B's column m is vals."""
    m = len(vals)
    n = m + 1
    colptr = np.concatenate([np.arange(n), [2 * m]]).astype(np.int64)
    rowidx = np.concatenate([np.arange(m), np.arange(m)]).astype(np.int32)
    return synth.CSC(n=n, colptr=colptr, rowidx=rowidx, val=np.concatenate([np.ones(m), vals]))


def _gpu_like(A, rows, vals, r=2.0):
    n = A.n
    rows = np.array(sorted(rows), np.int32)
    v = np.asarray(vals)[rows] ** r
    cp = np.zeros(n + 1, np.int64)
    cp[n] = len(rows)
    return synth.CSC(n=n, colptr=cp, rowidx=rows, val=v / v.sum())


def test_tie_at_the_recovery_cut_is_ambiguous_and_a_real_swap_is_not():
    vals = np.array([0.3, 0.2, 0.15, 0.1, 0.09, 0.08 * (1 + 1e-8), 0.08, 0.0])
    vals[-1] = 1.0 - vals[:-1].sum()
    A = _column_case(vals)
    j = np.array([A.n - 1], np.int32)
    prm = oracle.Params(theta=0.5, K=8, p=0.9)  # the recovery mass sets the cut
    res = oracle.expand_cols(A, prm, cols=j, topcap=8, kcap=8)
    kept = set(res.out_rows[0, :res.mstar[0]].tolist())
    assert kept == {0, 1, 2, 3, 4, 5}
    # rows 5 and 6 differ by 1e-8 relative (equal in FP32): either may be kept
    rep, _ = compare_iteration(A, _gpu_like(A, (kept - {5}) | {6}, vals), prm, cols=j)
    assert rep.ok() and rep.ambiguous_entries == 2
    # rows 4 and 6 differ by 12%: a swap is a real difference
    rep, _ = compare_iteration(A, _gpu_like(A, (kept - {4}) | {6}, vals), prm, cols=j)
    assert not rep.ok()
    # the oracle's own set passes
    rep, _ = compare_iteration(A, _gpu_like(A, kept, vals), prm, cols=j)
    assert rep.ok() and rep.ambiguous_entries == 0
