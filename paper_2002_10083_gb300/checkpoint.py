"""Checkpoint / resume of an MCL run.

Algorithm 1's whole state between iterations is the current matrix A_t,
the iteration count and the chaos history, so a run can stop after any
iteration and continue later: ``run`` iterates ``mcl_expand`` (through the
context) until chaos < eps or max_iters, writing that state to an ``.npz``
file every ``every`` iterations, and, when the file already exists,
continues from it.  The clusters are the connected components of the final
matrix (``mcl_components``).  Every step of an iteration runs in the
library; this module only moves the state between the device and a file.

The result equals an uninterrupted run's: the iteration only depends on
A_t (the learned sizing, when used, only changes how the numeric pass is
tiled, never its output).
"""
from __future__ import annotations

import json
import os

import numpy as np

FORMAT = 1


def save(path: str, A_host, iteration: int, chaos_hist, meta: dict | None = None) -> None:
    """Write the state after `iteration` iterations (atomically: temp file, then rename)."""
    tmp = path + ".tmp.npz"
    np.savez(tmp, format=FORMAT, n=A_host.n, colptr=A_host.colptr, rowidx=A_host.rowidx,
             val=A_host.val, iteration=iteration, chaos=np.asarray(chaos_hist, np.float64),
             meta=json.dumps(meta or {}))
    os.replace(tmp, path)


def load(path: str):
    """(A_host, iteration, chaos history, meta) of a checkpoint."""
    from .synth import CSC
    z = np.load(path)
    if int(z["format"]) != FORMAT:
        raise ValueError(f"checkpoint format {int(z['format'])} is not {FORMAT}")
    A = CSC(n=int(z["n"]), colptr=z["colptr"], rowidx=z["rowidx"], val=z["val"])
    return A, int(z["iteration"]), list(z["chaos"]), json.loads(str(z["meta"]))


def run(ctx, A0, prm, path: str, every: int = 1, stop_after: int | None = None,
        device_csc=None):
    """Algorithm 1 with a checkpoint every `every` iterations.

    A0: host CSC (used when `path` does not exist yet).  stop_after: return
    after this many iterations of this call (the state is saved), as a run
    that is interrupted would.  Returns (labels or None, iterations, chaos
    history, final device matrix, converged).
    """
    if device_csc is None:
        from .mcl import DeviceCSC as device_csc
    if os.path.exists(path):
        A, it, hist, _ = load(path)
    else:
        A, it, hist = A0, 0, []
    D = device_csc.from_host(A)
    done_here = 0
    converged = bool(hist) and hist[-1] < prm.chaos_eps
    while not converged and it < prm.max_iters:
        if stop_after is not None and done_here >= stop_after:
            return None, it, hist, D, False
        D, ch = ctx.expand(D, prm)
        hist.append(float(ch))
        it += 1
        done_here += 1
        converged = ch < prm.chaos_eps
        if it % every == 0 or converged or it == prm.max_iters:
            save(path, D.to_host(), it, hist, {"max_iters": prm.max_iters})
    labels = ctx.components(D)
    return labels, it, hist, D, converged
