"""Seeded synthetic inputs for the MCL expansion path.

This module only builds input graphs; it holds none of the method's
arithmetic (no expansion, pruning, inflation or chaos).  Both the CPU oracle
(test infrastructure) and the CUDA path consume the arrays it returns, so
one seeded call gives both sides identical inputs.

The paper's protein-similarity networks (Table I: archaea, eukarya,
isom100-*, metaclust50) are not available; these generators stand in for
their shape: power-law degrees, mean degree tens to hundreds, weighted,
symmetric, with self-loops, column-normalised as the first line of
Algorithm 1 requires ("column stochastic version of the weighted adjacency
matrix").

Recipes (all weights symmetric, one draw per undirected edge):

* ``planted_partition``: clusters of given sizes; each intra-cluster pair is
  an edge with probability ``p_in``, each inter-cluster pair with ``p_out``
  (exact Bernoulli per pair via geometric skipping); weights U(lo, hi].
* ``chung_lu``: target degrees w_i ~ discrete Zipf(a) truncated to
  [d_min, d_max]; ``round(sum(w)/2)`` edges with both endpoints drawn with
  probability proportional to w; self-pairs and duplicates dropped;
  weights lognormal(0, 1).
* ``component_batch``: block-diagonal union of planted partitions whose
  sizes are log-uniform, the batched workload.
* ``cliques``: block-diagonal uniform cliques (powers of two), an exact
  fixed point of MCL with inflation 2.

Self-loops: each vertex gets a loop whose weight is the largest
off-diagonal weight in its column (1.0 for an isolated vertex), added before
the column normalisation.  The paper says only that the matrix is column
stochastic; the loop weight is a reading, selectable with ``loop``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BASE_SEED = 2002


@dataclasses.dataclass
class CSC:
    """Compressed sparse column matrix with FP64 values (host arrays).

    colptr: int64[n+1]; rowidx: int32[nnz], strictly increasing per column;
    val: float64[nnz].  ``comp_offsets`` (optional int32[ncomp+1]) lists the
    first vertex of each independent component of a block-diagonal batch.
    """

    n: int
    colptr: np.ndarray
    rowidx: np.ndarray
    val: np.ndarray
    comp_offsets: np.ndarray | None = None
    labels: np.ndarray | None = None  # planted cluster id per vertex, if any

    @property
    def nnz(self) -> int:
        return int(self.colptr[-1])

    def val32(self) -> np.ndarray:
        return self.val.astype(np.float32)

    def with_val32(self) -> "CSC":
        """Copy whose values are the FP32-rounded values (as float64)."""
        return dataclasses.replace(self, val=self.val.astype(np.float32).astype(np.float64))


def rng_for(seed: int, stream: int = 0) -> np.random.Generator:
    """Philox stream keyed by (base seed, seed, stream)."""
    return np.random.Generator(np.random.Philox(key=[BASE_SEED ^ (seed & 0xFFFFFFFF), stream]))


# ---------------------------------------------------------------------------
# edge sampling helpers
# ---------------------------------------------------------------------------

def _bernoulli_positions(rng: np.random.Generator, m: int, p: float) -> np.ndarray:
    """Sorted positions in [0, m) each selected independently with prob p."""
    if m <= 0 or p <= 0.0:
        return np.zeros(0, dtype=np.int64)
    if p >= 1.0:
        return np.arange(m, dtype=np.int64)
    lam = math.log1p(-p)
    out = []
    pos = -1
    while True:
        want = int((m - pos) * p * 1.05) + 64
        u = rng.random(want)
        gaps = np.floor(np.log1p(-u) / lam).astype(np.int64) + 1
        cs = pos + np.cumsum(gaps)
        out.append(cs[cs < m])
        if cs[-1] >= m:
            break
        pos = int(cs[-1])
    return np.concatenate(out)


def _tri_unrank(lin: np.ndarray):
    """Linear index over pairs (i<j), ordered by j then i -> (i, j)."""
    lin = lin.astype(np.int64)
    j = np.floor((1.0 + np.sqrt(1.0 + 8.0 * lin.astype(np.float64))) / 2.0).astype(np.int64)
    # fix rounding: need j(j-1)/2 <= lin < j(j+1)/2
    for _ in range(3):
        lo = j * (j - 1) // 2
        j = np.where(lo > lin, j - 1, j)
        hi = j * (j + 1) // 2
        j = np.where(hi <= lin, j + 1, j)
    i = lin - j * (j - 1) // 2
    return i, j


def planted_partition_edges(rng, sizes, p_in, p_out):
    """Undirected edge list (i<j) of a planted partition with given cluster sizes."""
    sizes = np.asarray(sizes, dtype=np.int64)
    starts = np.concatenate([[0], np.cumsum(sizes)])
    n = int(starts[-1])
    ei, ej = [], []
    # intra-cluster pairs with p_in
    for c, s in enumerate(sizes):
        s = int(s)
        if s < 2:
            continue
        pos = _bernoulli_positions(rng, s * (s - 1) // 2, p_in)
        i, j = _tri_unrank(pos)
        ei.append(i + starts[c])
        ej.append(j + starts[c])
    # inter-cluster pairs with p_out: draw over all pairs, keep cross pairs
    if n >= 2 and p_out > 0:
        pos = _bernoulli_positions(rng, n * (n - 1) // 2, p_out)
        i, j = _tri_unrank(pos)
        ci = np.searchsorted(starts, i, side="right") - 1
        cj = np.searchsorted(starts, j, side="right") - 1
        keep = ci != cj
        ei.append(i[keep])
        ej.append(j[keep])
    if ei:
        return np.concatenate(ei), np.concatenate(ej), n
    return np.zeros(0, np.int64), np.zeros(0, np.int64), n


def zipf_degrees(rng, n, a, d_min, d_max):
    d = np.arange(d_min, d_max + 1, dtype=np.float64)
    pmf = d ** (-a)
    cdf = np.cumsum(pmf)
    cdf /= cdf[-1]
    u = rng.random(n)
    return d[np.searchsorted(cdf, u, side="right").clip(0, len(d) - 1)]


def zipf_dmin_for_mean(a, d_max, mean):
    """Smallest-error integer d_min giving the truncated Zipf law the mean."""
    best = None
    for dmin in range(1, d_max):
        d = np.arange(dmin, d_max + 1, dtype=np.float64)
        p = d ** (-a)
        m = float((d * p).sum() / p.sum())
        if best is None or abs(m - mean) < abs(best[1] - mean):
            best = (dmin, m)
        if m > mean * 1.5:
            break
    return best[0]


def _sorted_unique(k: np.ndarray) -> np.ndarray:
    k = np.sort(k)
    if len(k) == 0:
        return k
    keep = np.empty(len(k), dtype=bool)
    keep[0] = True
    np.not_equal(k[1:], k[:-1], out=keep[1:])
    return k[keep]


def chung_lu_edges(rng, n, a=2.0, mean=50.0, d_max=5000, d_min=None, chunk=1 << 24):
    """Chung-Lu edge list (i<j, deduplicated, no self pairs).

    Endpoints are drawn with probability proportional to w by picking a
    degree class (probability ~ d * count_d) and then a uniform member.
    """
    if d_min is None:
        d_min = zipf_dmin_for_mean(a, d_max, mean)
    w = zipf_degrees(rng, n, a, d_min, d_max)
    order = np.argsort(w, kind="stable")
    ws = w[order]
    cls_val, cls_start, cls_cnt = np.unique(ws, return_index=True, return_counts=True)
    cls_cdf = np.cumsum(cls_val * cls_cnt)
    total = float(cls_cdf[-1])
    m = int(round(total / 2.0))

    def draw(c):
        u = rng.random(c) * total
        cl = np.searchsorted(cls_cdf, u, side="right").clip(0, len(cls_val) - 1)
        v = rng.random(c)
        off = np.minimum((v * cls_cnt[cl]).astype(np.int64), cls_cnt[cl] - 1)
        return order[cls_start[cl] + off].astype(np.int64)

    keys = []
    done = 0
    while done < m:
        c = min(chunk, m - done)
        i = draw(c)
        j = draw(c)
        lo = np.minimum(i, j)
        hi = np.maximum(i, j)
        sel = lo != hi
        keys.append(hi[sel] * n + lo[sel])
        done += c
    k = _sorted_unique(np.concatenate(keys))
    ej = k // n
    ei = k - ej * n
    return ei, ej, w


# ---------------------------------------------------------------------------
# assembly: symmetric weighted graph -> column-stochastic CSC
# ---------------------------------------------------------------------------

def assemble(n, ei, ej, w, loop="max"):
    """Symmetric W (+ self-loops) -> A0 = W D^-1 in CSC with FP64 values.

    (ei, ej) are distinct undirected pairs with ei != ej, w the weight of
    each pair.  Loop weight: 'max' = largest off-diagonal weight in the
    column (1.0 if none), 'one' = 1.0, 'none' = no loops.
    """
    ei = np.asarray(ei, dtype=np.int64)
    ej = np.asarray(ej, dtype=np.int64)
    w = np.asarray(w, dtype=np.float64)
    lo = np.minimum(ei, ej)
    hi = np.maximum(ei, ej)
    pk = hi * n + lo                      # pair key; also the (col=hi,row=lo) entry key
    if len(pk) > 1 and not np.all(pk[1:] > pk[:-1]):
        o = np.argsort(pk, kind="stable")
        pk, lo, hi, w = pk[o], lo[o], hi[o], w[o]
    keys = np.sort(np.concatenate([pk, lo * n + hi]))   # key = col * n + row
    cols = keys // n
    rows = keys - cols * n
    pair = np.maximum(rows, cols) * n + np.minimum(rows, cols)
    vals = w[np.searchsorted(pk, pair)] if len(pk) else np.zeros(0)
    counts = np.bincount(cols, minlength=n).astype(np.int64)
    if loop != "none":
        if loop == "max":
            lw = np.ones(n, dtype=np.float64)
            nzc = counts > 0
            starts = np.concatenate([[0], np.cumsum(counts)[:-1]])
            if len(vals):
                mx = np.maximum.reduceat(vals, starts[nzc])
                lw[nzc] = mx
        elif loop == "one":
            lw = np.ones(n, dtype=np.float64)
        else:
            raise ValueError(loop)
        diag = np.arange(n, dtype=np.int64)
        pos = np.searchsorted(keys, diag * n + diag)
        keys = np.insert(keys, pos, diag * n + diag)
        vals = np.insert(vals, pos, lw)
        cols = keys // n
        rows = keys - cols * n
        counts = counts + 1
    colptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=colptr[1:])
    colsum = np.bincount(cols, weights=vals, minlength=n).astype(np.float64)
    nz = colsum > 0
    scale = np.where(nz, 1.0 / np.where(nz, colsum, 1.0), 0.0)
    vals = vals * scale[cols]
    return CSC(n=n, colptr=colptr, rowidx=rows.astype(np.int32), val=vals)


# ---------------------------------------------------------------------------
# the workloads
# ---------------------------------------------------------------------------

def planted_partition(n_clusters=20, cluster_size=100, p_in=0.1, p_out=0.001,
                      w_lo=0.5, w_hi=1.0, seed=0, loop="max"):
    """Planted partition graph, weights U(w_lo, w_hi]; 2,000 vertices by default."""
    rng = rng_for(seed, 1)
    sizes = [cluster_size] * n_clusters
    ei, ej, n = planted_partition_edges(rng, sizes, p_in, p_out)
    w = w_hi - (w_hi - w_lo) * rng.random(len(ei))  # in (lo, hi]
    A = assemble(n, ei, ej, w, loop=loop)
    A.labels = np.repeat(np.arange(n_clusters, dtype=np.int32), cluster_size)
    return A


def chung_lu(n=1_000_000, a=2.0, mean=50.0, d_max=5000, seed=0, loop="max"):
    """Power-law protein-similarity-shaped graph, lognormal(0,1) weights."""
    rng = rng_for(seed, 2)
    ei, ej, _ = chung_lu_edges(rng, n, a=a, mean=mean, d_max=d_max)
    w = rng.lognormal(0.0, 1.0, len(ei))
    return assemble(n, ei, ej, w, loop=loop)


def component_sizes(rng, ncomp, lo, hi):
    return np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi + 1), ncomp))).astype(np.int64).clip(lo, hi)


def component_batch(ncomp=4096, size_lo=50, size_hi=50000, c_lo=5, c_hi=200,
                    p_in=0.05, p_out=0.0005, w_lo=0.1, w_hi=1.0, seed=0, loop="max"):
    """Block-diagonal batch of planted partitions (the batched workload).

    Component sizes are log-uniform in [size_lo, size_hi]; each has c
    clusters, c uniform in [c_lo, c_hi] clamped to [2, size // 10], with
    sizes split as evenly as possible.
    """
    rng = rng_for(seed, 3)
    sizes = component_sizes(rng, ncomp, size_lo, size_hi)
    offs = np.zeros(ncomp + 1, dtype=np.int64)
    np.cumsum(sizes, out=offs[1:])
    all_i, all_j, labels = [], [], []
    lab0 = 0
    for c in range(ncomp):
        s = int(sizes[c])
        k = int(rng.integers(c_lo, c_hi + 1))
        k = max(2, min(k, s // 10))
        base, extra = divmod(s, k)
        csz = [base + (1 if q < extra else 0) for q in range(k)]
        ei, ej, _ = planted_partition_edges(rng, csz, p_in, p_out)
        all_i.append(ei + offs[c])
        all_j.append(ej + offs[c])
        labels.append(np.repeat(np.arange(k, dtype=np.int64) + lab0, csz))
        lab0 += k
    ei = np.concatenate(all_i)
    ej = np.concatenate(all_j)
    n = int(offs[-1])
    w = w_hi - (w_hi - w_lo) * rng.random(len(ei))
    A = assemble(n, ei, ej, w, loop=loop)
    A.comp_offsets = offs.astype(np.int32)
    A.labels = np.concatenate(labels).astype(np.int32)
    return A


def cliques(sizes, loop="one"):
    """Block-diagonal uniform cliques with loops: A0 = blockdiag(J/m)."""
    sizes = list(sizes)
    starts = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    ei, ej = [], []
    for c, m in enumerate(sizes):
        i, j = np.triu_indices(m, 1)
        ei.append(i + starts[c])
        ej.append(j + starts[c])
    ei = np.concatenate(ei) if ei else np.zeros(0, np.int64)
    ej = np.concatenate(ej) if ej else np.zeros(0, np.int64)
    A = assemble(int(starts[-1]), ei, ej, np.ones(len(ei)), loop=loop)
    A.labels = np.repeat(np.arange(len(sizes), dtype=np.int32), sizes)
    return A


def random_sparse(n, density, seed=0, loop="max", symmetric=True, w="uniform"):
    """Small random symmetric graph for unit tests."""
    rng = rng_for(seed, 4)
    pos = _bernoulli_positions(rng, n * (n - 1) // 2, density)
    ei, ej = _tri_unrank(pos)
    if w == "uniform":
        ww = 1.0 - rng.random(len(ei))
    elif w == "lognormal":
        ww = rng.lognormal(0.0, 1.0, len(ei))
    elif w == "one":
        ww = np.ones(len(ei))
    else:
        raise ValueError(w)
    return assemble(n, ei, ej, ww, loop=loop)


def random_csc(n_rows, n_cols, density, seed=0, lo=0.0, hi=1.0, empty_cols=()):
    """Random nonnegative CSC (not stochastic) for prune/inflate unit tests."""
    rng = rng_for(seed, 5)
    colptr = np.zeros(n_cols + 1, dtype=np.int64)
    rows, vals = [], []
    for j in range(n_cols):
        if j in empty_cols:
            r = np.zeros(0, dtype=np.int64)
        else:
            r = np.nonzero(rng.random(n_rows) < density)[0]
        rows.append(r)
        vals.append(lo + (hi - lo) * (1.0 - rng.random(len(r))))
        colptr[j + 1] = colptr[j] + len(r)
    return CSC(n=n_rows, colptr=colptr,
               rowidx=np.concatenate(rows).astype(np.int32) if rows else np.zeros(0, np.int32),
               val=np.concatenate(vals) if vals else np.zeros(0))


def config(name: str, seed: int = 0, **kw) -> CSC:
    """The named workloads (sizes as stated in each generator's docstring)."""
    if name == "planted2k":
        return planted_partition(seed=seed, **kw)
    if name == "zipf1m":
        return chung_lu(n=kw.pop("n", 1_000_000), mean=50.0, d_max=5000, seed=seed, **kw)
    if name == "batch4096":
        return component_batch(seed=seed, **kw)
    if name == "zipf4m":
        return chung_lu(n=kw.pop("n", 4_000_000), mean=120.0, d_max=5000, seed=seed, **kw)
    raise KeyError(name)
