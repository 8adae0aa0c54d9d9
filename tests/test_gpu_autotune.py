"""The autotuner on the GPU: every setting it tries gives the default's
result, and the winner is applied to the context."""
import numpy as np
import pytest
import torch

from paper_2002_10083_gb300 import autotune, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2002_10083_gb300 import mcl
    c = mcl.Context(0)
    yield c
    c.close()


def test_tune_small_power_law_graph(ctx, tmp_path):
    from paper_2002_10083_gb300 import mcl
    A = synth.chung_lu(n=40000, mean=40.0, d_max=2000, seed=3).with_val32()
    D = mcl.DeviceCSC.from_host(A)
    prm = mcl.Params(threshold=1e-4, select_k=300, recover_pct=0.9, inflation=2.0)
    try:
        res = autotune.tune(ctx, D, prm, reps=1)
        assert all(t["same"] for t in res["trials"]), res["trials"]
        assert len(res["trials"]) >= 7
        tried = {t["setting"]["table"] for t in res["trials"]}
        assert tried == {0, 1, 2}
        assert res["best_ms"] <= res["default_ms"]
        path = str(tmp_path / "t.json")
        wc = autotune.class_of_host(A)
        autotune.save(autotune.record({}, "dev", wc, res), path)
        got = autotune.apply(ctx, autotune.load(path), "dev", wc)
        assert got == res["best"]
        out, _ = ctx.expand(D, prm)
        assert out.nnz > 0
    finally:
        autotune.set_tuning(ctx, autotune.DEFAULTS)
