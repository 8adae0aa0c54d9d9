"""Plain FP64 CPU oracle for the MCL expansion path.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The product path never imports,
calls or links anything here, and nothing here imports the product path
(the seeded generators in ``paper_2002_10083_gb300.synth`` hold no method
arithmetic and are the only shared module).

The arithmetic lives in ``mcl_oracle.c`` (expansion, prune, inflation,
chaos, components; see its header for the passages each step follows) and
in ``mlp.py`` (the estimator network in FP64).  This module compiles the C
file with gcc and wraps it with ctypes, and adds the MCL loop of
Algorithm 1 on top.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mcl_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libmcl_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP over columns)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            i64 = ctypes.c_int64
            d = ctypes.c_double
            i = ctypes.c_int
            L.orc_expand_cols.argtypes = [i64, P, P, P, i64, P, d, i64, d, i64, d, i, i64, i64,
                                          P, P, P, P, P, P, P, P, P, P, i]
            L.orc_expand_cols.restype = i
            L.orc_prune_cols.argtypes = [P, P, P, i64, P, d, i64, d, i64, i64, P, P, P, P]
            L.orc_prune_cols.restype = i
            L.orc_inflate_normalize.argtypes = [i64, P, P, d, P]
            L.orc_inflate_normalize.restype = None
            L.orc_chaos.argtypes = [i64, P, P, P]
            L.orc_chaos.restype = None
            L.orc_symbolic_cols.argtypes = [i64, P, P, i64, P, P, P, i]
            L.orc_symbolic_cols.restype = i
            L.orc_components.argtypes = [i64, P, P, P]
            L.orc_components.restype = None
            L.orc_num_threads.argtypes = [i]
            L.orc_num_threads.restype = i
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads(nthreads: int = 0) -> int:
    return int(lib().orc_num_threads(nthreads))


@dataclasses.dataclass
class Params:
    """Prune / inflation parameters (threshold, top-k, recovery, inflation)."""
    theta: float = 1e-4
    K: int = 1100
    p: float = 0.9
    K_rec: int | None = None     # None -> K
    r: float = 2.0
    eps: float = 1e-3            # convergence threshold on chaos
    max_iters: int = 30

    @property
    def krec(self) -> int:
        return self.K if self.K_rec is None else self.K_rec


@dataclasses.dataclass
class ColumnResult:
    cols: np.ndarray
    flops: np.ndarray
    bnnz: np.ndarray
    bsum: np.ndarray
    ntop: np.ndarray
    top_rows: np.ndarray   # [ncols, topcap]
    top_vals: np.ndarray
    mstar: np.ndarray
    out_rows: np.ndarray   # [ncols, kcap]
    out_vals: np.ndarray
    chaos: np.ndarray
    kcap: int
    topcap: int


def _csc_arrays(A):
    colptr = np.ascontiguousarray(A.colptr, dtype=np.int64)
    rowidx = np.ascontiguousarray(A.rowidx, dtype=np.int32)
    val = np.ascontiguousarray(A.val, dtype=np.float64)
    return colptr, rowidx, val


def expand_cols(A, prm: Params, cols=None, inflate=True, topcap=0, kcap=None,
                nthreads=0) -> ColumnResult:
    """One MCL iteration restricted to the listed columns (all by default)."""
    colptr, rowidx, val = _csc_arrays(A)
    n = A.n
    cols = np.arange(n, dtype=np.int32) if cols is None else np.ascontiguousarray(cols, np.int32)
    m = len(cols)
    if kcap is None:
        kcap = max(1, min(n, max(prm.K, prm.krec)))
    topcap = int(topcap)
    f = np.zeros(m, np.int64)
    bn = np.zeros(m, np.int64)
    bs = np.zeros(m, np.float64)
    nt = np.zeros(m, np.int64)
    tr = np.zeros((m, max(topcap, 1)), np.int32)
    tv = np.zeros((m, max(topcap, 1)), np.float64)
    ms = np.zeros(m, np.int64)
    orow = np.zeros((m, kcap), np.int32)
    oval = np.zeros((m, kcap), np.float64)
    ch = np.zeros(m, np.float64)
    st = lib().orc_expand_cols(n, _p(colptr), _p(rowidx), _p(val), m, _p(cols), prm.theta,
                               int(prm.K), prm.p, int(prm.krec), prm.r, int(bool(inflate)),
                               topcap, kcap, _p(f), _p(bn), _p(bs), _p(nt), _p(tr), _p(tv),
                               _p(ms), _p(orow), _p(oval), _p(ch), int(nthreads))
    if st != 0:
        raise RuntimeError(f"oracle expand failed ({st})")
    return ColumnResult(cols, f, bn, bs, nt, tr, tv, ms, orow, oval, ch, kcap, topcap)


def result_to_csc(res: ColumnResult, n: int):
    """Assemble the kept columns of a full-matrix ColumnResult into a CSC."""
    from paper_2002_10083_gb300.synth import CSC
    assert len(res.cols) == n and np.all(res.cols == np.arange(n))
    colptr = np.zeros(n + 1, np.int64)
    np.cumsum(res.mstar, out=colptr[1:])
    mask = np.arange(res.kcap)[None, :] < res.mstar[:, None]
    return CSC(n=n, colptr=colptr, rowidx=res.out_rows[mask].astype(np.int32),
               val=res.out_vals[mask].astype(np.float64))


def expand(A, prm: Params, nthreads=0):
    """Full iteration: (A_next as CSC with FP64 values, chaos, ColumnResult)."""
    res = expand_cols(A, prm, nthreads=nthreads)
    An = result_to_csc(res, A.n)
    chaos = float(res.chaos.max()) if A.n else 0.0
    return An, chaos, res


def prune_cols(B, prm: Params, cols=None, kcap=None):
    """The prune rule alone on a given matrix (kept rows sorted, B values)."""
    colptr, rowidx, val = _csc_arrays(B)
    ncol = len(colptr) - 1
    cols = np.arange(ncol, dtype=np.int32) if cols is None else np.ascontiguousarray(cols, np.int32)
    m = len(cols)
    if kcap is None:
        kcap = max(1, int(np.diff(colptr).max(initial=1)))
    bs = np.zeros(m, np.float64)
    ms = np.zeros(m, np.int64)
    orow = np.zeros((m, kcap), np.int32)
    oval = np.zeros((m, kcap), np.float64)
    st = lib().orc_prune_cols(_p(colptr), _p(rowidx), _p(val), m, _p(cols), prm.theta,
                              int(prm.K), prm.p, int(prm.krec), kcap, _p(bs), _p(ms), _p(orow),
                              _p(oval))
    if st != 0:
        raise RuntimeError(f"oracle prune failed ({st})")
    return ms, orow, oval, bs


def inflate_normalize(A, r: float):
    """Inflation + column renormalisation of a copy of A; returns (A', chaos per column)."""
    colptr, rowidx, val = _csc_arrays(A)
    v = val.copy()
    ncol = len(colptr) - 1
    ch = np.zeros(ncol, np.float64)
    lib().orc_inflate_normalize(ncol, _p(colptr), _p(v), float(r), _p(ch))
    return dataclasses.replace(A, val=v), ch


def chaos_cols(A) -> np.ndarray:
    colptr, rowidx, val = _csc_arrays(A)
    ncol = len(colptr) - 1
    ch = np.zeros(ncol, np.float64)
    lib().orc_chaos(ncol, _p(colptr), _p(val), _p(ch))
    return ch


def chaos(A) -> float:
    ch = chaos_cols(A)
    return float(ch.max()) if len(ch) else 0.0


def symbolic_cols(A, cols=None, nthreads=0):
    """(flops_j, nnz(B_*j)) for the listed columns."""
    colptr, rowidx, _ = _csc_arrays(A)
    cols = np.arange(A.n, dtype=np.int32) if cols is None else np.ascontiguousarray(cols, np.int32)
    m = len(cols)
    f = np.zeros(m, np.int64)
    bn = np.zeros(m, np.int64)
    st = lib().orc_symbolic_cols(A.n, _p(colptr), _p(rowidx), m, _p(cols), _p(f), _p(bn),
                                 int(nthreads))
    if st != 0:
        raise RuntimeError("oracle symbolic failed")
    return f, bn


def components(A) -> np.ndarray:
    """Connected components of the undirected pattern; label = min vertex id."""
    colptr, rowidx, _ = _csc_arrays(A)
    lab = np.zeros(A.n, np.int32)
    lib().orc_components(A.n, _p(colptr), _p(rowidx), _p(lab))
    return lab


def run_mcl(A0, prm: Params, nthreads=0, per_component=None):
    """Algorithm 1: iterate expansion/prune/inflation until chaos < eps.

    Returns (A_final, iterations, chaos history, cluster labels).  With
    ``per_component`` (offsets of independent diagonal blocks), each block
    is iterated to its own convergence: a block whose chaos has dropped
    below eps is no longer expanded.
    """
    from paper_2002_10083_gb300.synth import CSC
    if per_component is not None:
        offs = np.asarray(per_component, np.int64)
        blocks, iters_all, hist_all = [], [], []
        for c in range(len(offs) - 1):
            sub = submatrix(A0, int(offs[c]), int(offs[c + 1]))
            Af, it, hist, _ = run_mcl(sub, prm, nthreads=nthreads)
            blocks.append((int(offs[c]), Af))
            iters_all.append(it)
            hist_all.append(hist)
        Af = block_diag(blocks, A0.n)
        return Af, iters_all, hist_all, components(Af)
    A = A0
    hist = []
    it = 0
    while it < prm.max_iters:
        A, ch, _ = expand(A, prm, nthreads=nthreads)
        it += 1
        hist.append(ch)
        if ch < prm.eps:
            break
    return A, it, hist, components(A)


def submatrix(A, lo: int, hi: int):
    """Diagonal block [lo, hi) of a block-diagonal CSC (rows re-based)."""
    from paper_2002_10083_gb300.synth import CSC
    s, e = int(A.colptr[lo]), int(A.colptr[hi])
    rows = A.rowidx[s:e].astype(np.int64)
    if len(rows) and (rows.min() < lo or rows.max() >= hi):
        raise ValueError("not block diagonal")
    return CSC(n=hi - lo, colptr=(A.colptr[lo:hi + 1] - s).astype(np.int64),
               rowidx=(rows - lo).astype(np.int32), val=A.val[s:e].copy())


def block_diag(blocks, n):
    from paper_2002_10083_gb300.synth import CSC
    colptr = np.zeros(n + 1, np.int64)
    rows, vals = [], []
    for lo, B in blocks:
        colptr[lo + 1:lo + B.n + 1] = np.diff(B.colptr)
        rows.append(B.rowidx.astype(np.int64) + lo)
        vals.append(B.val)
    np.cumsum(colptr, out=colptr)
    return CSC(n=n, colptr=colptr, rowidx=np.concatenate(rows).astype(np.int32),
               val=np.concatenate(vals))


def dense(A) -> np.ndarray:
    """Dense FP64 copy (tiny matrices only)."""
    ncol = len(A.colptr) - 1
    M = np.zeros((A.n, ncol), np.float64)
    for j in range(ncol):
        s, e = A.colptr[j], A.colptr[j + 1]
        M[A.rowidx[s:e], j] = A.val[s:e]
    return M
