"""Host logic of the autotuner (no GPU): workload classes, candidate
settings, and the stored table's round trip."""
import os

from paper_2002_10083_gb300 import autotune


class FakeCtx:
    def __init__(self):
        self.opts = {}

    def set_option(self, k, v):
        self.opts[k] = v


def test_workload_class_buckets():
    assert autotune.workload_class(1_000_000, 49_452_272, 5001) == "n19-mean5-max12"
    assert autotune.workload_class(1 << 20, 50 << 20, 4096) == "n20-mean5-max12"
    assert autotune.workload_class(0, 0, 0) == "n0-mean0-max0"


def test_candidates_cover_each_knob():
    best = dict(autotune.DEFAULTS)
    assert {c["table"] for c in autotune.candidates("table", best)} == {0, 1, 2}
    plans = [c["plan"] for c in autotune.candidates("plan", dict(best, table=1))]
    assert plans == [1024, 1536, 2048, 2560]
    assert all(p <= 0.75 * 4096 for p in plans)
    plans0 = [c["plan"] for c in autotune.candidates("plan", dict(best, table=0))]
    assert plans0 == [512, 768, 1024, 1280]
    assert {c["small_max"] for c in autotune.candidates("small_max", best)} == {0, 256, 512}


def test_table_round_trip_and_apply(tmp_path):
    path = os.path.join(tmp_path, "t.json")
    res = {"best": {"table": 2, "plan": 1536, "small_max": 256}, "best_ms": 1.5, "default_ms": 2.0}
    tab = autotune.record(autotune.load(path), "NVIDIA GB300", "n19-mean5-max12", res)
    autotune.save(tab, path)
    back = autotune.load(path)
    assert autotune.lookup(back, "NVIDIA GB300", "n19-mean5-max12") == res["best"]
    assert autotune.lookup(back, "other", "n19-mean5-max12") is None
    ctx = FakeCtx()
    got = autotune.apply(ctx, back, "NVIDIA GB300", "n19-mean5-max12")
    assert got == res["best"]
    assert ctx.opts == {autotune.OPT_TABLE: 2, autotune.OPT_PLAN: 1536, autotune.OPT_SMALL_MAX: 256}
    assert autotune.apply(FakeCtx(), back, "NVIDIA GB300", "n1-mean1-max1") is None


class _Csc:
    def __init__(self, colptr, rowidx, val):
        import torch
        self.colptr = torch.tensor(colptr, dtype=torch.int64)
        self.rowidx = torch.tensor(rowidx, dtype=torch.int32)
        self.val = torch.tensor(val, dtype=torch.float32)


def test_same_result_check_is_bitwise():
    pytest = __import__("pytest")
    pytest.importorskip("torch")
    n = 2000
    colptr = [2 * j for j in range(n + 1)]
    rows = [r for j in range(n) for r in (j, j + 1)]
    vals = [0.75, 0.25] * n
    ref = _Csc(colptr, rows, vals)
    ref.n = out_n = n
    same = _Csc(colptr, rows, vals)
    same.n = out_n
    assert autotune._same(same, ref)
    # one value one ulp away
    import numpy as np
    v1 = list(vals)
    v1[3] = float(np.nextafter(np.float32(v1[3]), np.float32(1.0)))
    other = _Csc(colptr, rows, v1)
    other.n = out_n
    assert not autotune._same(other, ref)
    # one row moved
    rows2 = list(rows)
    rows2[1] = 7
    other = _Csc(colptr, rows2, vals)
    other.n = out_n
    assert not autotune._same(other, ref)
