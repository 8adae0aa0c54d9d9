"""Pins of the FP64 CPU oracle against facts fixed by the paper and by the
mathematics (not against the oracle itself).

* expansion == dense numpy matmul on tiny inputs (Alg. 1, B <- AA);
* flops == sum_k nnz(A_*k)^2 for a symmetric pattern (Section II notation);
* column sums of A^2 are 1 for column-stochastic A; sums are 1 after every
  normalisation;
* the prune rule on hand-derived cases and on special cases that reduce to
  a plain sort / mask / cumulative sum;
* inflation at r = 0.5 ... 5 on hand-derived columns (tests/golden/inflate_cases.txt);
* chaos closed forms;
* planted cliques are an exact fixed point, recovered after one iteration;
* components == scipy's connected_components; vertex relabelling commutes.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2002_10083_gb300 import synth


def _read_cases(path):
    out = []
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        out.append([part.split() for part in line.split("|")])
    return out


def _one_col(rows, vals):
    rows = np.asarray(rows, np.int64)
    vals = np.asarray(vals, np.float64)
    o = np.argsort(rows)
    n = int(rows.max()) + 1 if len(rows) else 1
    return synth.CSC(n=n, colptr=np.array([0, len(rows)], np.int64),
                     rowidx=rows[o].astype(np.int32), val=vals[o])


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("n,dens", [(8, 0.5), (24, 0.2), (64, 0.08)])
def test_expansion_equals_dense_matmul(seed, n, dens):
    A = synth.random_sparse(n, dens, seed=seed, w="lognormal")
    prm = oracle.Params(theta=0.0, K=n + 1, p=1.0)
    res = oracle.expand_cols(A, prm, inflate=False)
    B = oracle.result_to_csc(res, n)
    D = oracle.dense(A)
    np.testing.assert_allclose(oracle.dense(B), D @ D, rtol=0, atol=1e-14)
    # nnz(B_*j) is the structural pattern of the boolean product
    P = (D != 0).astype(np.int64)
    assert np.array_equal(res.bnnz, ((P @ P) != 0).sum(0))
    # flops for a symmetric pattern: sum_j sum_{k in col j} nnz(col k) = sum_k d_k^2
    d = np.diff(A.colptr)
    assert res.flops.sum() == int((d.astype(np.int64) ** 2).sum())
    assert np.array_equal(res.flops, (P * d[:, None]).sum(0))
    # column sums of A^2 equal 1 for a column-stochastic A
    np.testing.assert_allclose(res.bsum, 1.0, rtol=0, atol=1e-12)


def test_expansion_nonsymmetric_against_matmul():
    # a non-symmetric pattern (as after pruning): still B = A A
    A = synth.random_csc(30, 30, 0.2, seed=3, lo=0.1, hi=1.0)
    D = oracle.dense(A)
    res = oracle.expand_cols(A, oracle.Params(theta=0.0, K=100, p=1.0), inflate=False)
    B = oracle.result_to_csc(res, 30)
    np.testing.assert_allclose(oracle.dense(B), D @ D, rtol=0, atol=1e-13)


def test_prune_golden_cases(golden_dir):
    cases = _read_cases(os.path.join(golden_dir, "prune_cases.txt"))
    assert len(cases) >= 8
    for (par, rows, vals, want) in cases:
        theta, K, p, Krec = float(par[0]), int(par[1]), float(par[2]), int(par[3])
        B = _one_col([int(r) for r in rows], [float(v) for v in vals])
        ms, orow, oval, _ = oracle.prune_cols(B, oracle.Params(theta=theta, K=K, p=p, K_rec=Krec),
                                              kcap=len(rows))
        got = sorted(orow[0, :ms[0]].tolist())
        assert got == sorted(int(w) for w in want), (par, rows, vals, got, want)


def _rand_col(rng, m):
    rows = np.sort(rng.choice(1000, size=m, replace=False))
    vals = rng.random(m)
    # a few exact ties
    if m > 3:
        vals[1] = vals[2]
    return rows, vals


def _value_order(rows, vals):
    return np.lexsort((rows, -vals))


@pytest.mark.parametrize("seed", range(20))
def test_prune_special_cases(seed):
    rng = np.random.default_rng(seed)
    m = int(rng.integers(1, 21))
    rows, vals = _rand_col(rng, m)
    B = _one_col(rows, vals)
    order = _value_order(rows, vals)
    K = int(rng.integers(1, m + 2))
    # theta = 0, K >= nnz, p = 1: identity
    ms, orow, oval, _ = oracle.prune_cols(B, oracle.Params(theta=0.0, K=m, p=1.0), kcap=m)
    assert ms[0] == m and np.array_equal(orow[0, :m], rows)
    np.testing.assert_array_equal(oval[0, :m], vals)
    # p = 0, theta = 0: pure top-K by (value desc, row asc)
    ms, orow, _, _ = oracle.prune_cols(B, oracle.Params(theta=0.0, K=K, p=0.0), kcap=m)
    assert sorted(orow[0, :ms[0]]) == sorted(rows[order[:min(K, m)]])
    # p = 0, K >= m: threshold mask b >= theta
    theta = float(np.quantile(vals, 0.5))
    ms, orow, _, _ = oracle.prune_cols(B, oracle.Params(theta=theta, K=m, p=0.0), kcap=m)
    assert sorted(orow[0, :ms[0]]) == sorted(rows[vals >= theta])
    # nothing reaches theta, K >= m: recovery alone = shortest value-sorted
    # prefix whose cumulative sum reaches p * sum
    p = float(rng.random())
    cs = np.cumsum(vals[order])
    need = int(np.searchsorted(cs, p * vals.sum(), side="left")) + 1
    need = 0 if p * vals.sum() <= 0 else min(need, m)
    ms, orow, _, _ = oracle.prune_cols(B, oracle.Params(theta=10.0, K=m, p=p), kcap=m)
    assert sorted(orow[0, :ms[0]]) == sorted(rows[order[:need]])


@pytest.mark.parametrize("seed", range(30))
def test_prune_properties(seed):
    """General case: kept set is a value-sorted prefix whose length obeys
    each constraint of the rule (select cap, threshold floor, recovery)."""
    rng = np.random.default_rng(100 + seed)
    m = int(rng.integers(1, 25))
    rows, vals = _rand_col(rng, m)
    theta = float(rng.random() * 0.8)
    K = int(rng.integers(1, m + 3))
    Krec = int(rng.integers(1, m + 3))
    p = float(rng.random())
    B = _one_col(rows, vals)
    ms, orow, _, _ = oracle.prune_cols(B, oracle.Params(theta=theta, K=K, p=p, K_rec=Krec), kcap=m)
    kept = set(orow[0, :ms[0]].tolist())
    order = _value_order(rows, vals)
    L = len(kept)
    assert kept == set(rows[order[:L]].tolist())          # a top prefix
    assert L <= min(Krec, m)                               # never above K_rec
    t = int((vals >= theta).sum())
    if L < Krec and L < m:
        assert L >= min(t, K)                              # threshold survivors up to K kept
        assert vals[order[:L]].sum() >= p * vals.sum() - 1e-15   # recovery reached
    if L > min(t, K):                                      # grown only by recovery: minimal
        assert vals[order[:L - 1]].sum() < p * vals.sum()


def test_chaos_golden(golden_dir):
    for vals, want in _read_cases(os.path.join(golden_dir, "chaos_cases.txt")):
        v = [float(x) for x in vals]
        A = _one_col(list(range(len(v))), v)
        assert abs(oracle.chaos_cols(A)[0] - float(want[0])) < 1e-15


def _inflate_cases(golden_dir):
    out = []
    for r, vals, want in _read_cases(os.path.join(golden_dir, "inflate_cases.txt")):
        num = [float(x) for x in want[:-2]]
        assert want[-2] == "/"
        out.append((float(r[0]), [float(v) for v in vals], np.array(num) / float(want[-1])))
    return out


def test_inflation_golden_cases(golden_dir):
    """Inflation at r != 1 against hand-derived columns (a wrong exponent,
    e.g. 1/r or r - 1, or a skipped power fails here)."""
    cases = _inflate_cases(golden_dir)
    assert len(cases) >= 8 and any(r not in (1.0, 2.0) for r, _, _ in cases)
    for r, vals, want in cases:
        A = _one_col(list(range(len(vals))), vals)
        out, ch = oracle.inflate_normalize(A, r)
        np.testing.assert_allclose(out.val, want, rtol=1e-14, atol=0, err_msg=f"r={r} {vals}")
        # chaos of the inflated column: max a - sum a^2
        assert abs(ch[0] - max(0.0, want.max() - (want ** 2).sum())) < 1e-15


def test_inflation_golden_cases_through_expansion(golden_dir):
    """The same columns as the last column of B = A A: columns 0..m-1 of A
    are unit vectors e_i, column m holds the case's values, so B's column m
    equals it; theta = 0, K >= m, p = 1 keep every entry, and the iteration
    returns the inflated, renormalised column."""
    for r, vals, want in _inflate_cases(golden_dir):
        m = len(vals)
        colptr = np.concatenate([np.arange(m + 1), [2 * m]]).astype(np.int64)
        rowidx = np.concatenate([np.arange(m), np.arange(m)]).astype(np.int32)
        val = np.concatenate([np.ones(m), vals])
        A = synth.CSC(n=m + 1, colptr=colptr, rowidx=rowidx, val=val)
        res = oracle.expand_cols(A, oracle.Params(theta=0.0, K=m + 1, p=1.0, r=r),
                                 cols=np.array([m], np.int32), inflate=True)
        assert res.mstar[0] == m and res.bnnz[0] == m
        assert np.array_equal(res.out_rows[0, :m], np.arange(m))
        np.testing.assert_allclose(res.out_vals[0, :m], want, rtol=1e-14, atol=0,
                                   err_msg=f"r={r} {vals}")


@pytest.mark.parametrize("seed", range(4))
def test_inflation_r1_no_prune_is_identity(seed):
    A = synth.random_sparse(50, 0.1, seed=seed, w="lognormal")
    prm = oracle.Params(theta=0.0, K=51, p=1.0, r=1.0)
    res = oracle.expand_cols(A, prm, inflate=True)
    B = oracle.result_to_csc(oracle.expand_cols(A, prm, inflate=False), 50)
    An = oracle.result_to_csc(res, 50)
    Bn = B.val / np.repeat(np.add.reduceat(B.val, B.colptr[:-1]), np.diff(B.colptr))
    np.testing.assert_allclose(An.val, Bn, rtol=1e-14)


def test_sums_one_after_every_normalisation():
    A = synth.config("planted2k")
    prm = oracle.Params(theta=1e-4, K=100, p=0.9, max_iters=8)
    for _ in range(6):
        A, ch, res = oracle.expand(A, prm)
        s = np.add.reduceat(A.val, A.colptr[:-1])
        np.testing.assert_allclose(s, 1.0, rtol=0, atol=1e-12)
        assert (A.val > 0).all()
        # kept count never exceeds K and is never zero (b_jj >= a_jj^2 > 0)
        assert res.mstar.max() <= prm.K and res.mstar.min() >= 1


@pytest.mark.parametrize("sizes", [[4, 8, 16], [32, 64], [4] * 10, [64, 4, 32, 8]])
def test_planted_cliques_fixed_point(sizes):
    A = synth.cliques(sizes)
    D = oracle.dense(A)
    assert np.array_equal(D @ D, D)            # blockdiag(J/m) is idempotent, exactly
    prm = oracle.Params(theta=1e-4, K=max(sizes), p=0.9, max_iters=30)
    A1, ch, _ = oracle.expand(A, prm)
    assert ch == 0.0
    assert np.array_equal(oracle.dense(A1), D)
    Af, it, hist, lab = oracle.run_mcl(A, prm)
    assert it == 1 and hist == [0.0]
    starts = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    assert np.array_equal(lab, np.repeat(starts, sizes).astype(np.int32))


@pytest.mark.parametrize("seed", range(5))
def test_components_match_scipy(seed):
    sp = pytest.importorskip("scipy.sparse")
    csg = pytest.importorskip("scipy.sparse.csgraph")
    A = synth.random_csc(300, 300, 0.004, seed=seed)
    lab = oracle.components(A)
    M = sp.csc_matrix((np.ones(A.nnz), A.rowidx, A.colptr), shape=(300, 300))
    nc, ref = csg.connected_components(M, directed=True, connection="weak")
    # same partition, and each label is the smallest member
    for c in range(nc):
        members = np.nonzero(ref == c)[0]
        assert (lab[members] == members.min()).all()


def test_vertex_permutation_equivariance():
    A = synth.random_sparse(80, 0.08, seed=7, w="lognormal")
    rng = np.random.default_rng(0)
    perm = rng.permutation(80)
    D = oracle.dense(A)
    Dp = D[np.ix_(perm, perm)]
    # rebuild the permuted matrix as CSC
    cols, rows = np.nonzero(Dp.T)
    Ap = synth.CSC(n=80, colptr=np.concatenate([[0], np.cumsum(np.bincount(cols, minlength=80))]).astype(np.int64),
                   rowidx=rows.astype(np.int32), val=Dp.T[cols, rows])
    prm = oracle.Params(theta=1e-3, K=20, p=0.9)
    A1, _, _ = oracle.expand(A, prm)
    A1p, _, _ = oracle.expand(Ap, prm)
    # ties could break differently after relabelling; this input has none
    np.testing.assert_allclose(oracle.dense(A1)[np.ix_(perm, perm)], oracle.dense(A1p), rtol=1e-12, atol=0)


def test_subset_columns_match_full():
    A = synth.random_sparse(120, 0.05, seed=11, w="lognormal")
    prm = oracle.Params(theta=1e-3, K=15, p=0.8)
    full = oracle.expand_cols(A, prm, topcap=20)
    cols = np.array([5, 77, 3, 119, 0], np.int32)
    sub = oracle.expand_cols(A, prm, cols=cols, topcap=20)
    for c, j in enumerate(cols):
        assert sub.mstar[c] == full.mstar[j]
        assert np.array_equal(sub.out_rows[c, :sub.mstar[c]], full.out_rows[j, :full.mstar[j]])
        np.testing.assert_array_equal(sub.out_vals[c], full.out_vals[j])
        assert sub.chaos[c] == full.chaos[j]


def test_symbolic_matches_expand():
    A = synth.random_sparse(200, 0.05, seed=2)
    f, bn = oracle.symbolic_cols(A)
    res = oracle.expand_cols(A, oracle.Params())
    assert np.array_equal(f, res.flops) and np.array_equal(bn, res.bnnz)


def test_empty_columns():
    A = synth.random_csc(20, 20, 0.3, seed=1, empty_cols=(0, 5, 19))
    res = oracle.expand_cols(A, oracle.Params(theta=0.0, K=30, p=1.0), inflate=True)
    for j in (0, 5, 19):
        assert res.mstar[j] == 0 and res.bnnz[j] == 0 and res.chaos[j] == 0.0
