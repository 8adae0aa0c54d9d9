"""GPU-vs-oracle comparison of one MCL iteration (test helper).

The oracle is fed the same input the GPU saw (its FP32 values widened to
FP64).  Per column:

* kept patterns must be identical, except entries that are ambiguous
  because FP32 rounding may legitimately flip them: within ``rtol`` of the
  prune threshold, of the K-th largest value, of the value at the cut (the
  last kept or first dropped value in oracle order, whichever rule set the
  cut: two entries equal in FP32 are ranked by row), or whose cumulative
  mass (in oracle order, before or including the entry) is within ``rtol``
  of the recovery target p * s;
* values must agree to ``rtol`` relative.  Where an ambiguous entry made
  the kept sets differ, the expected values are the oracle's B values
  inflated and renormalised over the GPU's kept set.
"""
from __future__ import annotations

import dataclasses

import numpy as np

import oracle


@dataclasses.dataclass
class Report:
    columns: int = 0
    entries: int = 0
    max_rel_err: float = 0.0
    ambiguous_cols: int = 0
    ambiguous_entries: int = 0
    failures: list = dataclasses.field(default_factory=list)

    def ok(self) -> bool:
        return not self.failures


def _col(A, j):
    s, e = int(A.colptr[j]), int(A.colptr[j + 1])
    return A.rowidx[s:e].astype(np.int64), A.val[s:e].astype(np.float64)


def compare_iteration(A_in, G_out, prm: oracle.Params, cols=None, rtol=1e-5, inflate=True,
                      max_fail=20, nthreads=0) -> Report:
    """A_in: input (host CSC, FP32-representable values); G_out: the GPU output."""
    n = A_in.n
    cols = np.arange(n, dtype=np.int32) if cols is None else np.asarray(cols, np.int32)
    K = prm.K
    topcap = max(prm.krec, K) + 64
    res = oracle.expand_cols(A_in, prm, cols=cols, inflate=inflate, topcap=topcap,
                             kcap=max(1, min(n, prm.krec)), nthreads=nthreads)
    rep = Report()
    for c, j in enumerate(cols):
        rep.columns += 1
        g_rows, g_vals = _col(G_out, int(j))
        m = int(res.mstar[c])
        o_rows = res.out_rows[c, :m].astype(np.int64)
        o_vals = res.out_vals[c, :m]
        if len(g_rows) > 1 and np.any(np.diff(g_rows) <= 0):
            rep.failures.append((int(j), "gpu rows not strictly increasing"))
            continue
        if np.array_equal(g_rows, o_rows):
            exp = o_vals
        else:
            # every differing entry must be ambiguous
            nt = int(res.ntop[c])
            trows = res.top_rows[c, :nt].astype(np.int64)
            tvals = res.top_vals[c, :nt]
            pos = {int(r): i for i, r in enumerate(trows)}
            s = float(res.bsum[c])
            target = prm.p * s
            bK = tvals[K - 1] if nt >= K else None
            # the values on both sides of the oracle's cut
            b_cut = [tvals[x] for x in (m - 1, m) if 0 <= x < nt]
            cum_incl = np.cumsum(tvals)
            cum_before = cum_incl - tvals
            diff = set(g_rows.tolist()) ^ set(o_rows.tolist())
            bad = []
            for r in diff:
                i = pos.get(int(r))
                if i is None:
                    bad.append(int(r))
                    continue
                b = tvals[i]
                amb = abs(b - prm.theta) <= rtol * prm.theta
                if bK is not None:
                    amb = amb or abs(b - bK) <= rtol * bK
                for bc in b_cut:
                    amb = amb or abs(b - bc) <= rtol * bc
                if target > 0:
                    amb = amb or abs(cum_before[i] - target) <= rtol * target
                    amb = amb or abs(cum_incl[i] - target) <= rtol * target
                if not amb:
                    bad.append(int(r))
            if bad:
                rep.failures.append((int(j), f"non-ambiguous pattern difference rows {bad[:8]}"))
                if len(rep.failures) >= max_fail:
                    break
                continue
            rep.ambiguous_cols += 1
            rep.ambiguous_entries += len(diff)
            bv = np.array([tvals[pos[int(r)]] for r in g_rows], dtype=np.float64)
            if inflate:
                u = bv ** prm.r
                exp = u / u.sum() if u.sum() > 0 else u
            else:
                exp = bv
        if len(exp):
            rel = np.abs(g_vals - exp) / np.maximum(np.abs(exp), 1e-300)
            mx = float(rel.max())
            rep.max_rel_err = max(rep.max_rel_err, mx)
            rep.entries += len(exp)
            if mx > rtol:
                k = int(np.argmax(rel))
                rep.failures.append((int(j), f"value rel err {mx:.3e} at row {g_rows[k]} "
                                             f"(gpu {g_vals[k]!r} oracle {exp[k]!r})"))
                if len(rep.failures) >= max_fail:
                    break
    return rep, res
