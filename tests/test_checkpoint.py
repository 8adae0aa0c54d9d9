"""Checkpoint / resume logic on the CPU with a stand-in context whose
"iteration" is deterministic host arithmetic: an interrupted and resumed
run ends where an uninterrupted one does, with the same history."""
import dataclasses
import os

import numpy as np

from paper_2002_10083_gb300 import checkpoint
from paper_2002_10083_gb300.synth import CSC


@dataclasses.dataclass
class Prm:
    chaos_eps: float = 1e-3
    max_iters: int = 30


class HostCsc:
    """Host stand-in for DeviceCSC (from_host / to_host)."""

    def __init__(self, A):
        self.A = A

    @staticmethod
    def from_host(A):
        return HostCsc(CSC(n=A.n, colptr=np.array(A.colptr), rowidx=np.array(A.rowidx),
                           val=np.array(A.val, np.float32)))

    def to_host(self):
        return self.A


class FakeCtx:
    """Each 'iteration' halves every value's distance to its column mean;
    chaos = largest distance."""

    def __init__(self):
        self.calls = 0

    def expand(self, D, prm):
        self.calls += 1
        A = D.A
        v = A.val.astype(np.float64).copy()
        for j in range(A.n):
            s, e = A.colptr[j], A.colptr[j + 1]
            if e > s:
                m = v[s:e].mean()
                v[s:e] = m + (v[s:e] - m) / 2
        ch = 0.0
        for j in range(A.n):
            s, e = A.colptr[j], A.colptr[j + 1]
            if e > s:
                ch = max(ch, float(np.abs(v[s:e] - v[s:e].mean()).max()))
        return HostCsc(CSC(n=A.n, colptr=A.colptr, rowidx=A.rowidx, val=v.astype(np.float32))), ch

    def components(self, D):
        return np.arange(D.A.n, dtype=np.int32)


def _matrix():
    rng = np.random.default_rng(0)
    n = 20
    colptr = np.arange(0, 3 * n + 1, 3, dtype=np.int64)
    rowidx = np.array([(j + d) % n for j in range(n) for d in (0, 1, 2)], np.int32)
    return CSC(n=n, colptr=colptr, rowidx=rowidx, val=rng.random(3 * n).astype(np.float32))


def test_interrupted_run_resumes_to_the_same_end(tmp_path):
    A0 = _matrix()
    prm = Prm()
    full = str(tmp_path / "full.npz")
    lab, it, hist, D, conv = checkpoint.run(FakeCtx(), A0, prm, full, device_csc=HostCsc)
    assert conv and it == len(hist) and hist[-1] < prm.chaos_eps
    part = str(tmp_path / "part.npz")
    ctx1 = FakeCtx()
    lab1, it1, hist1, _, conv1 = checkpoint.run(ctx1, A0, prm, part, every=1, stop_after=3,
                                                device_csc=HostCsc)
    assert lab1 is None and it1 == 3 and not conv1 and os.path.exists(part)
    ctx2 = FakeCtx()
    lab2, it2, hist2, D2, conv2 = checkpoint.run(ctx2, A0, prm, part, device_csc=HostCsc)
    assert ctx2.calls == it - 3
    assert conv2 and it2 == it
    np.testing.assert_allclose(hist2, hist, rtol=0, atol=0)
    np.testing.assert_array_equal(D2.A.val, D.A.val)
    # a finished checkpoint resumes to no further work
    ctx3 = FakeCtx()
    _, it3, _, _, conv3 = checkpoint.run(ctx3, A0, prm, part, device_csc=HostCsc)
    assert ctx3.calls == 0 and it3 == it and conv3


def test_checkpoint_file_round_trip(tmp_path):
    A = _matrix()
    p = str(tmp_path / "c.npz")
    checkpoint.save(p, A, 7, [0.5, 0.25], {"k": 1})
    B, it, hist, meta = checkpoint.load(p)
    assert it == 7 and hist == [0.5, 0.25] and meta == {"k": 1}
    np.testing.assert_array_equal(B.colptr, A.colptr)
    np.testing.assert_array_equal(B.rowidx, A.rowidx)
    np.testing.assert_array_equal(B.val, A.val)
