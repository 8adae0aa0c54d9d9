"""FP64 oracle of Cohen's probabilistic output-size estimate (Section V).

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU leg).

The product A A is a three-layer graph: first-layer vertices are the rows
i of A, middle vertices the columns k of A (rows of the right factor), last
the columns j.  Each first-layer vertex gets r keys from Exp(lambda = 1);
the middle layer keeps, per key index, the minimum over its in-neighbours,
the last layer the minimum over its middle in-neighbours, and the estimate
of the number of first-layer vertices reaching j is (r - 1) / sum of its r
minimum keys.

Keys: splitmix64 (Steele, Lea and Flood 2014; the generator of Java's
SplittableRandom) evaluated at counter seed + (i * r + l) * 0x9E3779B97F4A7C15
(mod 2^64); u = (top 53 bits + 1) / 2^53 in (0, 1]; key = -ln(u).
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """One splitmix64 output for each 64-bit state x (state advanced once)."""
    with np.errstate(over="ignore"):
        z = (np.asarray(x, dtype=np.uint64) + GOLDEN).astype(np.uint64)
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)).astype(np.uint64)
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)).astype(np.uint64)
        return z ^ (z >> np.uint64(31))


def keys(n: int, r: int, seed: int) -> np.ndarray:
    """[n, r] keys -ln(u) in FP64."""
    i = np.arange(n, dtype=np.uint64)[:, None]
    l = np.arange(r, dtype=np.uint64)[None, :]
    with np.errstate(over="ignore"):
        ctr = (np.uint64(seed) + (i * np.uint64(r) + l) * GOLDEN).astype(np.uint64)
    z = splitmix64(ctr)
    u = ((z >> np.uint64(11)).astype(np.float64) + 1.0) / 9007199254740992.0
    return -np.log(u)


def _colmin(colptr, rowidx, vals_per_row):
    """min over each column's rows of vals_per_row[row] ([n, r]); inf if empty."""
    ncol = len(colptr) - 1
    r = vals_per_row.shape[1]
    out = np.full((ncol, r), np.inf)
    deg = np.diff(colptr)
    nz = np.nonzero(deg)[0]
    if len(nz):
        g = vals_per_row[np.asarray(rowidx, np.int64)]
        out[nz] = np.minimum.reduceat(g, np.asarray(colptr[:-1], np.int64)[nz], axis=0)
    return out


def estimate(A, r: int, seed: int) -> np.ndarray:
    """Cohen's estimate of nnz((AA)_*j) for every column j."""
    K = keys(A.n, r, seed)
    m = _colmin(A.colptr, A.rowidx, K)     # middle layer
    M = _colmin(A.colptr, A.rowidx, m)     # last layer
    S = M.sum(axis=1)
    with np.errstate(divide="ignore"):
        est = np.where(np.isfinite(S) & (S > 0), (r - 1) / S, 0.0)
    return est
