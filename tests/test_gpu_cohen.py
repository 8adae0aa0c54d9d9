"""GPU tests of Cohen's probabilistic output-size estimate (Section V)
through the C ABI: the per-column estimates against the FP64 oracle on the
same keys (same counter-based generator, each side its own), the
estimate against the exact symbolic counts, and the Cohen-sized expansion
against the oracle."""
import numpy as np
import pytest

import oracle
from oracle import cohen
from paper_2002_10083_gb300 import synth
from tests.parity import compare_iteration

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# keys in FP32 (a few ulp from -ln u) and an FP32 sum of at most 16 minima
RTOL = 1e-5


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2002_10083_gb300 import mcl
    c = mcl.Context(0)
    yield c
    c.close()


def _dev(A):
    from paper_2002_10083_gb300 import mcl
    return mcl.DeviceCSC.from_host(A)


@pytest.mark.parametrize("graph", ["random", "chung_lu", "batch"])
@pytest.mark.parametrize("r,seed", [(2, 0), (8, 2002), (16, 123456789012345)])
def test_cohen_matches_oracle(ctx, graph, r, seed):
    if graph == "random":
        A = synth.random_sparse(3000, 0.003, seed=1)
    elif graph == "chung_lu":
        A = synth.chung_lu(n=20000, mean=30.0, d_max=3000, seed=2)
    else:
        A = synth.component_batch(40, 20, 300, seed=3)
    A = A.with_val32()
    G = ctx.cohen_estimate(_dev(A), keys=r, seed=seed).cpu().numpy().astype(np.float64)
    O = cohen.estimate(A, r, seed)
    np.testing.assert_array_equal(G == 0, O == 0)
    np.testing.assert_allclose(G, O, rtol=RTOL, atol=0)


def test_cohen_empty_and_isolated_columns(ctx):
    # columns with no entries, and columns whose sources are all empty
    n = 6
    colptr = np.array([0, 0, 1, 1, 3, 3, 4], np.int64)
    rowidx = np.array([1, 0, 2, 3], np.int32)  # col1 -> {1}; col3 -> {0, 2}; col5 -> {3}
    A = synth.CSC(n=n, colptr=colptr, rowidx=rowidx, val=np.ones(4, np.float32))
    G = ctx.cohen_estimate(_dev(A), keys=5, seed=9).cpu().numpy().astype(np.float64)
    O = cohen.estimate(A, 5, 9)
    np.testing.assert_allclose(G, O, rtol=RTOL, atol=0)
    # col 0 is empty, col 3 reaches only empty columns
    assert G[0] == 0 and G[2] == 0 and G[3] == 0 and G[1] > 0 and G[5] > 0


def test_cohen_rejects_bad_key_count(ctx):
    from paper_2002_10083_gb300 import mcl
    D = _dev(synth.random_sparse(100, 0.05, seed=0).with_val32())
    for r in (0, 1, 17):
        with pytest.raises(mcl.MclError):
            ctx.cohen_estimate(D, keys=r)
    for v in (1, 17):
        with pytest.raises(mcl.MclError):
            ctx.set_option(mcl.OPT_COHEN_KEYS, v)


def test_cohen_estimates_the_symbolic_counts(ctx):
    """Per column, est_j / nnz_j is distributed as (r - 1) / Gamma(r, 1)
    (relative sd 1/sqrt(r - 2)); the total is within about 10% (Section
    VII-C).  Hub-free random graph, checked against the exact symbolic
    counts of the GPU symbolic pass."""
    from scipy import stats
    A = synth.random_sparse(50000, 0.0004, seed=31).with_val32()
    D = _dev(A)
    fl, nz = ctx.symbolic(D)
    nz = nz.double().cpu().numpy()
    for r in (8, 16):
        est = ctx.cohen_estimate(D, keys=r, seed=0).double().cpu().numpy()
        q = est / nz
        assert abs(est.sum() / nz.sum() - 1.0) < 0.10, (r, est.sum(), nz.sum())
        assert abs(np.median(q) / ((r - 1) / stats.gamma.ppf(0.5, r)) - 1.0) < 0.10
        assert 0.8 < np.std(q - 1.0) * np.sqrt(r - 2) < 1.2, (r, np.std(q - 1.0))


def test_cohen_total_on_a_power_law_graph(ctx):
    """On a hub-dominated graph most columns reach the same hubs and share
    their minimum keys, so the per-seed error of the total does not average
    out over columns (about 16% sd at r = 16); the mean over seeds is still
    unbiased."""
    A = synth.chung_lu(n=100000, mean=40.0, d_max=5000, seed=21).with_val32()
    D = _dev(A)
    fl, nz = ctx.symbolic(D)
    tot = float(nz.double().sum())
    for r in (8, 16):
        ratios = [float(ctx.cohen_estimate(D, keys=r, seed=s).double().sum()) / tot
                  for s in range(8)]
        assert abs(np.mean(ratios) - 1.0) < 0.10, (r, ratios)


@pytest.mark.parametrize("keys,scale", [(8, 1000), (4, 1000), (16, 300)])
def test_cohen_sizing_expansion_matches_oracle(ctx, keys, scale):
    """The Cohen-sized numeric pass (windows planned from the estimate, with
    misses caught by the overflow path) produces the oracle's iteration."""
    from paper_2002_10083_gb300 import mcl
    A = synth.chung_lu(n=20000, mean=60.0, d_max=2000, seed=5).with_val32()
    D = _dev(A)
    prm = mcl.Params(threshold=1e-4, select_k=300, recover_pct=0.9)
    try:
        ctx.set_option(mcl.OPT_SIZING, mcl.SIZING_COHEN)
        ctx.set_option(mcl.OPT_COHEN_KEYS, keys)
        ctx.set_option(mcl.OPT_EST_SCALE, scale)
        out, ch = ctx.expand(D, prm)
    finally:
        ctx.set_option(mcl.OPT_SIZING, -1)
        ctx.set_option(mcl.OPT_COHEN_KEYS, 8)
        ctx.set_option(mcl.OPT_EST_SCALE, 1000)
    G = out.to_host()
    cols = np.random.default_rng(4).choice(A.n, 600, replace=False).astype(np.int32)
    oprm = oracle.Params(theta=float(np.float32(1e-4)), K=300, p=float(np.float32(0.9)), r=2.0)
    rep, _ = compare_iteration(A, G, oprm, cols=cols, rtol=RTOL)
    assert rep.ok(), rep.failures[:5]
    ref, ch_ref = ctx.expand(D, prm)
    assert abs(out.nnz - ref.nnz) <= 1e-6 * ref.nnz
