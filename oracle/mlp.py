"""FP64 oracle of the learned output-size estimator (test infrastructure).

Only tests, the smoke check and the benchmark's CPU leg use this module.

Per-column features (16, FP64, listed in FEATURES) and a 16 -> 64 -> 64 -> 2
MLP with ReLU activations whose weights are given as BF16 bit patterns
(uint16); inputs are standardised with (x - mu) / sigma.  Outputs:
y0 = log(1 + nnz((AA)_*j)), y1 = log(flops_j / max(nnz_j, 1)) (the
compression factor cf of Section II's notation, in log).  The loss of a
batch of B samples is (1/B) * sum over samples and outputs of (y - t)^2.

Parameter layout (flat, 5378 values): W1 [64 x 16] (row = output unit),
b1 [64], W2 [64 x 64], b2 [64], W3 [2 x 64], b3 [2].
"""
from __future__ import annotations

import numpy as np

NIN, NH, NOUT = 16, 64, 2
SHAPES = [("W1", (NH, NIN)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)),
          ("W3", (NOUT, NH)), ("b3", (NOUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)
HUGE_DEG = 1024  # a referenced column counts as "huge" above this many entries

FEATURES = [
    "log1p(nnz_j)", "log1p(flops_j)", "log1p(max_k nnz_k)", "log1p(mean_k nnz_k)",
    "log1p(var_k nnz_k)", "max_k a_kj", "sum_k a_kj", "sum_k a_kj^2",
    "log1p(row span of column j)", "fraction of k with nnz_k > 1024", "log(n)",
    "log1p(iteration)", "previous log cf_j (0 if none)", "mean_k max value of column k",
    "log1p(row span of the product column)", "1",
]


def bf16_round_bits(x: np.ndarray) -> np.ndarray:
    """FP32 -> BF16 bit patterns, round to nearest even (NaN not expected)."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return r.astype(np.uint16)


def bf16_bits_to_f64(b: np.ndarray) -> np.ndarray:
    return (np.asarray(b, np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def unpack(theta: np.ndarray):
    out, o = {}, 0
    for name, shp in SHAPES:
        m = int(np.prod(shp))
        out[name] = theta[o:o + m].reshape(shp)
        o += m
    return out


def pack(parts: dict) -> np.ndarray:
    return np.concatenate([np.asarray(parts[name], np.float64).ravel() for name, _ in SHAPES])


def forward(theta, X, mu, sigma, keep=False):
    """theta: FP64 weights (already BF16 values); X: [B, 16]."""
    P = unpack(theta)
    Z = (np.asarray(X, np.float64) - mu) / sigma
    A1 = Z @ P["W1"].T + P["b1"]
    H1 = np.maximum(A1, 0.0)
    A2 = H1 @ P["W2"].T + P["b2"]
    H2 = np.maximum(A2, 0.0)
    Y = H2 @ P["W3"].T + P["b3"]
    if keep:
        return Y, (Z, A1, H1, A2, H2)
    return Y


def loss(theta, X, T, mu, sigma):
    Y = forward(theta, X, mu, sigma)
    return float(((Y - T) ** 2).sum() / len(X))


def grad(theta, X, T, mu, sigma):
    """Backpropagation of the batch loss; returns (loss, dtheta)."""
    P = unpack(theta)
    Y, (Z, A1, H1, A2, H2) = forward(theta, X, mu, sigma, keep=True)
    B = len(X)
    dY = 2.0 * (Y - T) / B
    g = {"W3": dY.T @ H2, "b3": dY.sum(0)}
    dH2 = dY @ P["W3"]
    dA2 = dH2 * (A2 > 0)
    g["W2"] = dA2.T @ H1
    g["b2"] = dA2.sum(0)
    dH1 = dA2 @ P["W2"]
    dA1 = dH1 * (A1 > 0)
    g["W1"] = dA1.T @ Z
    g["b1"] = dA1.sum(0)
    return float(((Y - T) ** 2).sum() / B), pack(g)


def column_features(A, iteration: int = 1, prev_logcf=None, cols=None) -> np.ndarray:
    """The 16 features of each listed column of A (host CSC), FP64."""
    n = A.n
    colptr = np.asarray(A.colptr, np.int64)
    rowidx = np.asarray(A.rowidx, np.int64)
    val = np.asarray(A.val, np.float64)
    deg = np.diff(colptr)
    first = np.where(deg > 0, rowidx[np.minimum(colptr[:-1], max(len(rowidx) - 1, 0))], 0) if len(rowidx) else np.zeros(n, np.int64)
    last = np.where(deg > 0, rowidx[np.maximum(colptr[1:] - 1, 0)], -1) if len(rowidx) else np.full(n, -1)
    colmax = np.zeros(n)
    for k in range(n):
        if deg[k]:
            colmax[k] = val[colptr[k]:colptr[k + 1]].max()
    cols = np.arange(n) if cols is None else np.asarray(cols)
    F = np.zeros((len(cols), NIN), np.float64)
    for c, j in enumerate(cols):
        s, e = colptr[j], colptr[j + 1]
        ks = rowidx[s:e]
        a = val[s:e]
        d = len(ks)
        dk = deg[ks].astype(np.float64)
        flops = dk.sum()
        F[c, 0] = np.log1p(d)
        F[c, 1] = np.log1p(flops)
        if d:
            F[c, 2] = np.log1p(dk.max())
            F[c, 3] = np.log1p(dk.mean())
            F[c, 4] = np.log1p(max(0.0, (dk * dk).mean() - dk.mean() ** 2))
            F[c, 5] = a.max()
            F[c, 6] = a.sum()
            F[c, 7] = (a * a).sum()
            F[c, 8] = np.log1p(ks[-1] - ks[0] + 1)
            F[c, 9] = (dk > HUGE_DEG).mean()
            F[c, 13] = colmax[ks].mean()
            nzk = deg[ks] > 0
            if nzk.any():
                F[c, 14] = np.log1p(last[ks][nzk].max() - first[ks][nzk].min() + 1)
        F[c, 10] = np.log(max(n, 1))
        F[c, 11] = np.log1p(iteration)
        F[c, 12] = 0.0 if prev_logcf is None else float(prev_logcf[j])
        F[c, 15] = 1.0
    return F
