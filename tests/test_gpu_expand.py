"""GPU parity tests of the fused MCL iteration and the standalone entry
points, through the C ABI, against the FP64 oracle fed the same input.

Tolerance: 1e-5 relative per value (FP32 values and accumulation against
FP64); kept patterns identical except ambiguous boundary entries (see
tests/parity.py).
"""
import numpy as np
import pytest

import oracle
from paper_2002_10083_gb300 import synth
from tests.parity import compare_iteration

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-5


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2002_10083_gb300 import mcl
    c = mcl.Context(0)
    yield c
    c.close()


def _prm(theta=1e-4, K=100, p=0.9, Krec=0, r=2.0, eps=1e-3, iters=30):
    from paper_2002_10083_gb300 import mcl
    return mcl.Params(threshold=theta, select_k=K, recover_pct=p, recover_k=Krec, inflation=r,
                      chaos_eps=eps, max_iters=iters)


def _oprm(p):
    return oracle.Params(theta=float(np.float32(p.threshold)), K=p.select_k,
                         p=float(np.float32(p.recover_pct)),
                         K_rec=p.recover_k if p.recover_k > 0 else None,
                         r=float(np.float32(p.inflation)), eps=p.chaos_eps, max_iters=p.max_iters)


def _dev(A):
    from paper_2002_10083_gb300 import mcl
    return mcl.DeviceCSC.from_host(A)


def _assert_same(out, ref):
    assert out.n == ref.n and out.nnz == ref.nnz
    assert torch.equal(out.colptr, ref.colptr) and torch.equal(out.rowidx, ref.rowidx)
    assert torch.equal(out.val.view(torch.int32), ref.val.view(torch.int32))


def _check(ctx, A, prm, cols=None):
    A32 = A.with_val32()
    D = _dev(A32)
    out, ch = ctx.expand(D, prm)
    torch.cuda.synchronize()
    G = out.to_host()
    rep, res = compare_iteration(A32, G, _oprm(prm), cols=cols, rtol=RTOL)
    assert rep.ok(), rep.failures[:5]
    if cols is None and A.n:
        och = float(res.chaos.max())
        # chaos_j <= max a; value errors of rtol bound its error by 3 rtol max a
        assert abs(ch - och) <= 3 * RTOL * max(1.0, och) + 1e-12, (ch, och)
    return rep, G, ch


@pytest.mark.parametrize("n,dens,seed", [(300, 0.03, 0), (1000, 0.01, 1), (3000, 0.004, 2),
                                         (777, 0.02, 3)])
@pytest.mark.parametrize("K,p,theta", [(100, 0.9, 1e-4), (20, 0.5, 1e-3), (1, 0.9, 1e-4),
                                       (4096, 1.0, 0.0), (64, 0.0, 0.0)])
def test_expand_random(ctx, n, dens, seed, K, p, theta):
    A = synth.random_sparse(n, dens, seed=seed, w="lognormal")
    rep, G, _ = _check(ctx, A, _prm(theta=theta, K=K, p=p))
    assert rep.entries > 0


@pytest.mark.parametrize("mask", [0b01, 0b10, 0b11])
@pytest.mark.parametrize("scale", [1000, 20])
def test_expand_multi_range_and_splits(ctx, mask, scale):
    """Columns far larger than one window: several row windows (mask 1 forces
    the small configuration on every column), and with a deliberate 50x
    under-estimate, window overflow + cutting."""
    from paper_2002_10083_gb300 import mcl
    A = synth.chung_lu(n=20000, mean=60.0, d_max=2000, seed=5)
    try:
        ctx.set_option(mcl.OPT_CONF_MASK, mask)
        ctx.set_option(mcl.OPT_EST_SCALE, scale)
        cols = np.random.default_rng(0).choice(A.n, 600, replace=False).astype(np.int32)
        rep, G, _ = _check(ctx, A, _prm(K=300, p=0.9), cols=cols)
        st = ctx.stats()
        if scale < 1000:
            assert st["range_splits"] > 0 and st["estimator_misses"] > 0
    finally:
        ctx.set_option(mcl.OPT_CONF_MASK, 0x3)
        ctx.set_option(mcl.OPT_EST_SCALE, 1000)


@pytest.mark.parametrize("sizing", [0, 1, 3])
def test_sizing_modes_same_result(ctx, sizing):
    from paper_2002_10083_gb300 import mcl
    A = synth.random_sparse(2000, 0.01, seed=9, w="lognormal").with_val32()
    D = _dev(A)
    try:
        ctx.set_option(mcl.OPT_SIZING, sizing)
        out, ch = ctx.expand(D, _prm(K=50))
    finally:
        ctx.set_option(mcl.OPT_SIZING, -1)
    ref, ch2 = ctx.expand(D, _prm(K=50))
    # fixed-point accumulation: the sizing only plans the windows, the result is bit-identical
    _assert_same(out, ref)
    assert ch == ch2


def test_planted2k_iterations_and_clusters(ctx):
    """The 2,000-vertex planted partition: every GPU iteration matches the
    oracle fed the GPU's own input; the clusters equal the oracle's run."""
    A = synth.config("planted2k").with_val32()
    prm = _prm(theta=1e-4, K=100, p=0.9, iters=30)
    D = _dev(A)
    it = 0
    host_in = A
    while it < prm.max_iters:
        out, ch = ctx.expand(D, prm)
        G = out.to_host()
        rep, res = compare_iteration(host_in, G, _oprm(prm), rtol=RTOL)
        assert rep.ok(), (it, rep.failures[:5])
        it += 1
        D, host_in = out, G
        if ch < prm.chaos_eps:
            break
    lab_gpu, iters, hist, final, notconv = ctx.run(_dev(A), prm)
    assert not notconv and iters == it
    _, o_iters, o_hist, o_lab = oracle.run_mcl(A, _oprm(prm))
    assert iters == o_iters
    assert np.array_equal(lab_gpu.cpu().numpy(), o_lab)


@pytest.mark.parametrize("sizes", [[4, 8, 16], [32, 64, 4, 8], [64] * 20])
def test_cliques_fixed_point(ctx, sizes):
    A = synth.cliques(sizes)
    prm = _prm(theta=1e-4, K=max(sizes), p=0.9)
    lab, iters, hist, final, notconv = ctx.run(_dev(A), prm)
    assert iters == 1 and hist[0] == 0.0
    starts = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    assert np.array_equal(lab.cpu().numpy(), np.repeat(starts, sizes))
    F = final.to_host()
    np.testing.assert_array_equal(F.val, A.val.astype(np.float32).astype(np.float64))


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("K,p,theta,Krec", [(5, 0.9, 0.3, 0), (1, 0.5, 0.0, 0), (8, 0.0, 0.2, 0),
                                            (3, 0.95, 0.9, 6), (4096, 1.0, 0.0, 0)])
def test_prune_standalone(ctx, seed, K, p, theta, Krec):
    B = synth.random_csc(400, 400, 0.05, seed=seed, lo=0.0, hi=1.0, empty_cols=(3, 17))
    # a column of exact ties
    B.val[B.colptr[5]:B.colptr[6]] = 0.25
    B32 = B.with_val32()
    prm = _prm(theta=theta, K=K, p=p, Krec=Krec)
    out = ctx.prune_select_recover(_dev(B32), prm)
    G = out.to_host()
    ms, orow, oval, _ = oracle.prune_cols(B32, _oprm(prm))
    for j in range(B.n):
        s, e = G.colptr[j], G.colptr[j + 1]
        assert e - s == ms[j], j
        assert np.array_equal(G.rowidx[s:e], orow[j, :ms[j]]), j
        np.testing.assert_array_equal(G.val[s:e], oval[j, :ms[j]])


def test_inflate_normalize_and_chaos_standalone(ctx):
    A = synth.random_csc(500, 500, 0.03, seed=4, lo=0.01, hi=2.0, empty_cols=(7,)).with_val32()
    D = _dev(A)
    ctx.inflate_normalize(D, 2.0)
    G = D.to_host()
    ref, och = oracle.inflate_normalize(A, 2.0)
    np.testing.assert_allclose(G.val, ref.val, rtol=RTOL, atol=0)
    ch, cols = ctx.chaos(D, per_column=True)
    gch = oracle.chaos_cols(G)
    np.testing.assert_allclose(cols.cpu().numpy(), gch, rtol=1e-12, atol=1e-15)
    assert abs(ch - gch.max()) <= 1e-15


def test_chaos_golden_columns(ctx, golden_dir):
    import os
    rows, vals, cp, want = [], [], [0], []
    for line in open(os.path.join(golden_dir, "chaos_cases.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        v, w = line.split("|")
        v = [float(x) for x in v.split()]
        rows += list(range(len(v)))
        vals += v
        cp.append(cp[-1] + len(v))
        want.append(float(w))
    n = max(len(cp) - 1, max(rows) + 1)
    cp += [cp[-1]] * (n + 1 - len(cp))
    A = synth.CSC(n=n, colptr=np.array(cp, np.int64), rowidx=np.array(rows, np.int32),
                  val=np.array(vals))
    ch, cols = ctx.chaos(_dev(A), per_column=True)
    c = cols.cpu().numpy()
    for i, w in enumerate(want):
        # FP32 inputs: a value like 0.9 is not exact in FP32
        assert abs(c[i] - w) < 1e-6, (i, c[i], w)


@pytest.mark.parametrize("seed", range(3))
def test_components(ctx, seed):
    A = synth.random_csc(5000, 5000, 0.0003, seed=seed)
    lab = ctx.components(_dev(A)).cpu().numpy()
    assert np.array_equal(lab, oracle.components(A))


def test_symbolic(ctx):
    A = synth.random_sparse(3000, 0.01, seed=3)
    fl, nz = ctx.symbolic(_dev(A))
    of, on = oracle.symbolic_cols(A)
    assert np.array_equal(fl.cpu().numpy(), of)
    assert np.array_equal(nz.cpu().numpy(), on)


def test_symbolic_windows_large_span(ctx):
    # spans above one bitmap window (524,288 rows) use several windows
    A = synth.chung_lu(n=700000, mean=8.0, d_max=500, seed=1)
    fl, nz = ctx.symbolic(_dev(A))
    cols = np.random.default_rng(1).choice(A.n, 3000, replace=False).astype(np.int32)
    of, on = oracle.symbolic_cols(A, cols=cols)
    assert np.array_equal(fl.cpu().numpy()[cols], of)
    assert np.array_equal(nz.cpu().numpy()[cols], on)


def test_edge_cases(ctx):
    from paper_2002_10083_gb300 import mcl
    prm = _prm(K=10)
    # n = 0
    E = synth.CSC(n=0, colptr=np.zeros(1, np.int64), rowidx=np.zeros(0, np.int32), val=np.zeros(0))
    out, ch = ctx.expand(_dev(E), prm)
    assert out.n == 0 and out.nnz == 0 and ch == 0.0
    # empty columns and a single entry
    A = synth.random_csc(50, 50, 0.1, seed=2, lo=0.1, hi=1.0, empty_cols=(0, 1, 49))
    _check(ctx, A, prm)
    # all-equal values: ties at the k-th value resolved by the smaller row
    A = synth.random_sparse(200, 0.1, seed=3, w="one", loop="one")
    _check(ctx, A, _prm(K=7, p=0.5))


@pytest.mark.parametrize("kind", ["order", "range", "value", "nan", "colptr"])
def test_invalid_input_rejected(ctx, kind):
    from paper_2002_10083_gb300 import mcl
    A = synth.random_sparse(100, 0.05, seed=1)
    rowidx = A.rowidx.copy()
    val = A.val.copy()
    colptr = A.colptr.copy()
    s = colptr[10]
    if kind == "order":
        rowidx[s], rowidx[s + 1] = rowidx[s + 1], rowidx[s]
    elif kind == "range":
        rowidx[colptr[20 + 1] - 1] = 100
    elif kind == "value":
        val[5] = -0.5
    elif kind == "nan":
        val[7] = np.nan
    elif kind == "colptr":
        colptr[30] = colptr[31] + 1
    B = synth.CSC(n=A.n, colptr=colptr, rowidx=rowidx, val=val)
    with pytest.raises(mcl.MclError) as ei:
        ctx.expand(_dev(B), _prm(K=10))
    assert ei.value.status == 1
    # the context stays usable
    _check(ctx, A, _prm(K=10))


def test_bad_params_rejected(ctx):
    from paper_2002_10083_gb300 import mcl
    A = _dev(synth.random_sparse(50, 0.1, seed=1))
    for bad in (dict(K=0), dict(K=5000), dict(p=1.5), dict(theta=-1.0), dict(r=0.0)):
        with pytest.raises(mcl.MclError):
            ctx.expand(A, _prm(**bad))


@pytest.fixture(scope="module")
def zipf1m():
    return synth.config("zipf1m").with_val32()


def test_zipf1m_one_iteration_sampled(ctx, zipf1m):
    """The 1M-vertex power-law workload at full size: sampled columns
    against the oracle, every output column sums to 1."""
    A = zipf1m
    prm = _prm(theta=1e-4, K=1100, p=0.9)
    D = _dev(A)
    out, ch = ctx.expand(D, prm)
    torch.cuda.synchronize()
    G = out.to_host()
    sums = np.add.reduceat(G.val, G.colptr[:-1]) if G.nnz else np.zeros(0)
    nzc = np.diff(G.colptr) > 0
    np.testing.assert_allclose(sums[nzc], 1.0, rtol=0, atol=2e-5)
    rng = np.random.default_rng(2002)
    deg = np.diff(A.colptr)
    cols = np.concatenate([rng.choice(A.n, 1500, replace=False),
                           np.argsort(-deg)[:40]]).astype(np.int32)  # include the hubs
    rep, res = compare_iteration(A, G, _oprm(prm), cols=cols, rtol=RTOL)
    assert rep.ok(), rep.failures[:5]
    st = ctx.stats()
    assert st["flops"] == int((deg.astype(np.int64) ** 2).sum())


@pytest.mark.slow
def test_zipf1m_iterations_2_and_3_sampled(ctx, zipf1m):
    """Iterations 2 and 3 of the 1M-vertex power-law workload, where the
    columns of the input hold up to K = 1,100 entries and the products per
    column reach about a million: each GPU iteration against the oracle fed
    the GPU's own input, on random columns plus the columns with the most
    products, and every output column sums to 1."""
    prm = _prm(theta=1e-4, K=1100, p=0.9)
    D = _dev(zipf1m)
    D, _ = ctx.expand(D, prm)  # iteration 1 (checked in the test above)
    for it in (2, 3):
        Hin = D.to_host()
        out, ch = ctx.expand(D, prm)
        torch.cuda.synchronize()
        G = out.to_host()
        sums = np.add.reduceat(G.val, G.colptr[:-1]) if G.nnz else np.zeros(0)
        nzc = np.diff(G.colptr) > 0
        np.testing.assert_allclose(sums[nzc], 1.0, rtol=0, atol=2e-5)
        deg = np.diff(Hin.colptr)
        fl = np.zeros(Hin.n, np.int64)
        np.add.at(fl, np.repeat(np.arange(Hin.n), deg), deg[Hin.rowidx])  # flops_j
        rng = np.random.default_rng(2002 + it)
        cols = np.unique(np.concatenate([rng.choice(Hin.n, 800, replace=False),
                                         np.argsort(-fl)[:40]])).astype(np.int32)
        rep, res = compare_iteration(Hin, G, _oprm(prm), cols=cols, rtol=RTOL)
        assert rep.ok(), (it, rep.failures[:5])
        assert ctx.stats()["flops"] == int(fl.sum())
        D = out


@pytest.mark.parametrize("seed", [0, 1])
def test_batched_components_match_per_component_runs(ctx, seed):
    """Batched MCL over independent components (each stops on its own chaos)
    equals running every component separately, on the GPU and in the
    oracle."""
    from paper_2002_10083_gb300 import mcl
    A = synth.component_batch(ncomp=24, size_lo=50, size_hi=1500, p_in=0.3, p_out=0.002,
                              seed=seed).with_val32()
    offs = A.comp_offsets
    prm = _prm(theta=1e-4, K=200, p=0.9, iters=40)
    prm.batched = 1
    lab, iters, hist, final, notconv = ctx.run(_dev(A), prm, comp_offsets=offs)
    assert not notconv
    lab = lab.cpu().numpy()
    # oracle, per component
    _, o_iters, _, o_lab = oracle.run_mcl(A, _oprm(prm), per_component=offs)
    assert iters == max(o_iters)
    assert np.array_equal(lab, o_lab)
    # GPU, per component, one run each
    prm1 = _prm(theta=1e-4, K=200, p=0.9, iters=40)
    for c in range(len(offs) - 1):
        sub = oracle.submatrix(A, int(offs[c]), int(offs[c + 1]))
        l1, it1, _, _, nc1 = ctx.run(_dev(sub), prm1, keep_final=False)
        assert it1 == o_iters[c]
        assert np.array_equal(l1.cpu().numpy() + offs[c], lab[offs[c]:offs[c + 1]])


def test_batched_rejects_non_block_diagonal(ctx):
    from paper_2002_10083_gb300 import mcl
    A = synth.random_sparse(100, 0.05, seed=1)
    prm = _prm()
    prm.batched = 1
    with pytest.raises(mcl.MclError) as ei:
        ctx.run(_dev(A), prm, comp_offsets=np.array([0, 50, 100], np.int32))
    assert ei.value.status == 1


@pytest.mark.parametrize("budget", [64 * 1024, 1 << 20])
def test_column_batched_expansion_equals_single_pass(ctx, budget):
    """Consecutive column batches whose output staging fits a budget (the
    phased expansion) give the same iteration as one pass."""
    from paper_2002_10083_gb300 import mcl
    A = synth.chung_lu(n=30000, mean=30.0, d_max=2000, seed=8).with_val32()
    D = _dev(A)
    prm = _prm(K=500, p=0.9)
    ref, ch_ref = ctx.expand(D, prm)
    try:
        ctx.set_option(mcl.OPT_PHASE_BUDGET, budget)
        out, ch = ctx.expand(D, prm)
        phases = ctx.stats()["phases"]
    finally:
        ctx.set_option(mcl.OPT_PHASE_BUDGET, 0)
    assert phases > 1
    _assert_same(out, ref)
    assert ch == ch_ref
    cols = np.random.default_rng(5).choice(A.n, 500, replace=False).astype(np.int32)
    rep, _ = compare_iteration(A, out.to_host(), _oprm(prm), cols=cols, rtol=RTOL)
    assert rep.ok(), rep.failures[:5]


@pytest.mark.parametrize("cap,learned,scale", [(0, False, 1000), (1, False, 1000),
                                               (0, True, 1000), (0, True, 20)])
def test_batched_graph_replay_matches_eager(ctx, cap, learned, scale):
    """Batched MCL with iterations after the first replayed as CUDA graphs
    gives the same iterations, clusters and chaos history as the eager
    loop; cap 1 shrinks the replay buffers below an iteration's capacities,
    so that the device guard stops the replay and the host finishes
    without graphs."""
    from paper_2002_10083_gb300 import mcl
    A = synth.component_batch(ncomp=16, size_lo=50, size_hi=1200, p_in=0.3, p_out=0.002,
                              seed=4).with_val32()
    offs = A.comp_offsets
    prm = _prm(theta=1e-4, K=200, p=0.9, iters=40)
    prm.batched = 1
    if learned:  # learned sizing: features and MLP inside the replayed graph
        from paper_2002_10083_gb300 import estimator
        estimator.install(ctx)
        prm.use_estimator = 1
    try:
        # scale 20: every learned estimate 50x too small, so that the run
        # falls back to exact sizing after the first iteration
        ctx.set_option(mcl.OPT_EST_SCALE, scale)
        ctx.set_option(mcl.OPT_GRAPH, 0)
        lab0, it0, hist0, _, nc0 = ctx.run(_dev(A), prm, comp_offsets=offs, keep_final=False)
        st0 = ctx.stats()
        assert st0["graph_replays"] == 0
        ctx.set_option(mcl.OPT_GRAPH, 1)
        ctx.set_option(mcl.OPT_GRAPH_CAP, cap)
        lab1, it1, hist1, _, nc1 = ctx.run(_dev(A), prm, comp_offsets=offs, keep_final=False)
        st1 = ctx.stats()
        replays = st1["graph_replays"]
    finally:
        ctx.set_option(mcl.OPT_GRAPH, 1)
        ctx.set_option(mcl.OPT_GRAPH_CAP, 0)
        ctx.set_option(mcl.OPT_EST_SCALE, 1000)
    if scale < 1000:
        assert st0["exact_from"] == 2 and st1["exact_from"] == 2
    assert not nc0 and not nc1
    assert it0 == it1 and it1 > 2
    assert replays >= 1
    if cap == 0:
        assert replays == it1 - 1
    assert np.array_equal(lab0.cpu().numpy(), lab1.cpu().numpy())
    # exact fixed-point accumulation: graph replays and the eager loop give the
    # same matrices bit for bit, so the same chaos history
    assert hist1[:it1] == hist0[:it0]
    # and the per-component oracle
    _, o_iters, _, o_lab = oracle.run_mcl(A, _oprm(prm), per_component=offs)
    assert it1 == max(o_iters)
    assert np.array_equal(lab1.cpu().numpy(), o_lab)


def test_batched_groups_equal_one_run(ctx):
    """A batch run in consecutive groups of whole components (a group budget
    far below the batch's needs) gives the single run's iterations, chaos
    history, clusters and final matrix, bit for bit."""
    from paper_2002_10083_gb300 import mcl
    A = synth.component_batch(ncomp=16, size_lo=50, size_hi=1200, p_in=0.3, p_out=0.002,
                              seed=6).with_val32()
    offs = A.comp_offsets
    prm = _prm(theta=1e-4, K=200, p=0.9, iters=40)
    prm.batched = 1
    lab0, it0, hist0, F0, nc0 = ctx.run(_dev(A), prm, comp_offsets=offs)
    assert ctx.stats()["groups"] == 1
    try:
        ctx.set_option(mcl.OPT_GROUP_BUDGET, 12 << 20)
        lab1, it1, hist1, F1, nc1 = ctx.run(_dev(A), prm, comp_offsets=offs)
        groups = ctx.stats()["groups"]
    finally:
        ctx.set_option(mcl.OPT_GROUP_BUDGET, 0)
    assert groups > 2
    assert not nc0 and not nc1 and it0 == it1 and hist0 == hist1
    assert np.array_equal(lab0.cpu().numpy(), lab1.cpu().numpy())
    _assert_same(F1, F0)
    _, o_iters, _, o_lab = oracle.run_mcl(A, _oprm(prm), per_component=offs)
    assert it1 == max(o_iters) and np.array_equal(lab1.cpu().numpy(), o_lab)


@pytest.mark.parametrize("graph", [0, 1])
def test_batched_flops_count_only_active_components(ctx, graph):
    """A batched run's multiply-adds are those of each component's own
    iterations up to and including the one where it converged (retired
    components are carried, not expanded), eager and as graph replays."""
    from paper_2002_10083_gb300 import mcl
    A = synth.component_batch(ncomp=8, size_lo=50, size_hi=600, p_in=0.3, p_out=0.002,
                              seed=9).with_val32()
    offs = A.comp_offsets
    prm = _prm(theta=1e-4, K=200, p=0.9, iters=40)
    prm.batched = 1
    try:
        ctx.set_option(mcl.OPT_GRAPH, graph)
        _, iters, _, _, nc = ctx.run(_dev(A), prm, comp_offsets=offs, keep_final=False)
        got = ctx.stats()["flops_run"]
    finally:
        ctx.set_option(mcl.OPT_GRAPH, 1)  # the library default
    assert not nc
    want, longest = 0, 0
    for c in range(len(offs) - 1):
        D = _dev(oracle.submatrix(A, int(offs[c]), int(offs[c + 1])))
        for it in range(iters):
            D, ch = ctx.expand(D, prm)
            want += ctx.stats()["flops"]
            if ch < prm.chaos_eps:
                break
        longest = max(longest, it + 1)
    assert longest == iters
    assert got == want


def test_batched_groups_wider_than_one_launch_grid(ctx):
    """Groups of 1.4M columns each (more than the 1,245,184 threads of a
    capped launch grid): every group's column pointers are re-based and
    placed back in full, and the result equals the single-group run.
    700,000 disjoint 4-cliques with uniform weights are a fixed point of the
    iteration, so the clusters are the cliques."""
    from paper_2002_10083_gb300 import mcl
    m, ncl = 4, 700_000
    n = m * ncl
    base = (np.arange(n, dtype=np.int64) // m) * m
    A = synth.CSC(n=n, colptr=np.arange(n + 1, dtype=np.int64) * m,
                  rowidx=(np.repeat(base, m) + np.tile(np.arange(m), n)).astype(np.int32),
                  val=np.full(n * m, 1.0 / m)).with_val32()
    offs = np.array([0, n // 2, n], np.int32)
    prm = _prm(theta=1e-4, K=100, p=0.9, iters=5)
    prm.batched = 1
    lab0, it0, _, F0, nc0 = ctx.run(_dev(A), prm, comp_offsets=offs)
    assert ctx.stats()["groups"] == 1
    try:
        ctx.set_option(mcl.OPT_GROUP_BUDGET, 6 << 30)
        lab1, it1, _, F1, nc1 = ctx.run(_dev(A), prm, comp_offsets=offs)
        groups = ctx.stats()["groups"]
    finally:
        ctx.set_option(mcl.OPT_GROUP_BUDGET, 0)
    assert groups == 2
    assert not nc0 and not nc1 and it0 == it1 == 1
    assert np.array_equal(lab1.cpu().numpy(), base.astype(np.int32))
    assert np.array_equal(lab0.cpu().numpy(), lab1.cpu().numpy())
    _assert_same(F1, F0)


@pytest.mark.parametrize("learned", [False, True])
def test_batched_graph_replay_every_iteration_matches_oracle(ctx, learned):
    """Every replayed iteration of a batched run against the oracle fed the
    same input.  Runs are bit-identical, so the run capped at t iterations
    returns exactly the A_t that the run capped at t + 1 iterations expanded
    in its replayed iteration t + 1: each component still active there must
    match the oracle's iteration of its block of A_t (1e-5 per value), and
    each retired component's columns must be carried over bit for bit."""
    from paper_2002_10083_gb300 import mcl
    A = synth.component_batch(ncomp=16, size_lo=50, size_hi=1200, p_in=0.3, p_out=0.002,
                              seed=4).with_val32()
    offs = A.comp_offsets
    prm = _prm(theta=1e-4, K=200, p=0.9, iters=40)
    prm.batched = 1
    if learned:
        from paper_2002_10083_gb300 import estimator
        estimator.install(ctx)
        prm.use_estimator = 1
    _, o_iters, _, _ = oracle.run_mcl(A, _oprm(prm), per_component=offs)
    T = min(6, max(o_iters))
    mats = {}
    for t in range(1, T + 1):
        prm.max_iters = t
        _, it, _, final, _ = ctx.run(_dev(A), prm, comp_offsets=offs)
        assert it == min(t, max(o_iters))
        if t >= 2:
            assert ctx.stats()["graph_replays"] == t - 1
        mats[t] = final.to_host()
    checked = 0
    for t in range(1, T):
        At, At1 = mats[t], mats[t + 1]
        for c in range(len(offs) - 1):
            lo, hi = int(offs[c]), int(offs[c + 1])
            sub_in = oracle.submatrix(At, lo, hi)
            sub_out = oracle.submatrix(At1, lo, hi)
            if t < o_iters[c]:  # component c is expanded in iteration t + 1
                rep, _ = compare_iteration(sub_in, sub_out, _oprm(prm), rtol=RTOL)
                assert rep.ok(), (t + 1, c, rep.failures[:3])
                checked += 1
            else:  # retired: carried unchanged
                assert np.array_equal(sub_in.colptr, sub_out.colptr)
                assert np.array_equal(sub_in.rowidx, sub_out.rowidx)
                assert np.array_equal(sub_in.val, sub_out.val)
    assert checked >= T - 1


@pytest.mark.slow
def test_zipf4m_degree_law_column_batched_sampled():
    """The 4M-vertex workload's degree law (Zipf(2), mean 120, capped at
    5,000) at a quarter of its vertices, expanded in column batches under a
    small staging budget: sampled columns (the hubs included) against the
    oracle, every output column sums to 1."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2002_10083_gb300 import estimator, mcl
    A = synth.config("zipf4m", n=1_000_000).with_val32()
    ctx = mcl.Context(0)
    try:
        estimator.install(ctx)
        ctx.set_option(mcl.OPT_PHASE_BUDGET, 2 << 30)
        prm = _prm(theta=1e-4, K=1100, p=0.9)
        prm.use_estimator = 1
        out, ch = ctx.expand(_dev(A), prm)
        assert ctx.stats()["phases"] > 1
        torch.cuda.synchronize()
        G = out.to_host()
    finally:
        ctx.close()
    sums = np.add.reduceat(G.val, G.colptr[:-1]) if G.nnz else np.zeros(0)
    nzc = np.diff(G.colptr) > 0
    np.testing.assert_allclose(sums[nzc], 1.0, rtol=0, atol=2e-5)
    deg = np.diff(A.colptr)
    rng = np.random.default_rng(2004)
    cols = np.concatenate([rng.choice(A.n, 600, replace=False),
                           np.argsort(-deg)[:20]]).astype(np.int32)
    rep, _ = compare_iteration(A, G, _oprm(prm), cols=cols, rtol=RTOL)
    assert rep.ok(), rep.failures[:5]


def _host_ram_gb():
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemTotal:"):
                return int(line.split()[1]) / 2 ** 20
    except OSError:
        pass
    return 0.0


@pytest.mark.slow
def test_zipf4m_iterations_1_and_2_full_size_sampled():
    """The 4M-vertex workload at its stated size, as configured (learned
    sizing, column batches under a 180 GB staging budget): iterations 1 and
    2 against the oracle fed the GPU's own input on 20,000 random columns
    each (plus the 40 with the most products), and every output column sums
    to 1."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    if _host_ram_gb() < 160:
        pytest.skip("needs about 160 GB of host memory for the oracle's copy of A_1")
    from paper_2002_10083_gb300 import estimator, mcl
    A = synth.config("zipf4m").with_val32()
    ctx = mcl.Context(0)
    try:
        estimator.install(ctx)
        ctx.set_option(mcl.OPT_PHASE_BUDGET, 180 << 30)
        prm = _prm(theta=1e-4, K=1100, p=0.9)
        prm.use_estimator = 1
        D = _dev(A)
        Hin = A
        for it in (1, 2):
            ctx.set_option(mcl.OPT_ITERATION, it)
            out, ch = ctx.expand(D, prm)
            torch.cuda.synchronize()
            G = out.to_host()
            sums = np.add.reduceat(G.val, G.colptr[:-1]) if G.nnz else np.zeros(0)
            nzc = np.diff(G.colptr) > 0
            np.testing.assert_allclose(sums[nzc], 1.0, rtol=0, atol=2e-5)
            deg = np.diff(Hin.colptr)
            fl = np.zeros(Hin.n, np.int64)
            np.add.at(fl, np.repeat(np.arange(Hin.n), deg), deg[Hin.rowidx])
            rng = np.random.default_rng(4000 + it)
            cols = np.unique(np.concatenate([rng.choice(Hin.n, 20000, replace=False),
                                             np.argsort(-fl)[:40]])).astype(np.int32)
            rep, _ = compare_iteration(Hin, G, _oprm(prm), cols=cols, rtol=RTOL)
            assert rep.ok(), (it, rep.failures[:5])
            assert ctx.stats()["flops"] == int(fl.sum())
            del D
            D, Hin = out, G
    finally:
        ctx.close()


def test_checkpointed_run_equals_mcl_run(ctx, tmp_path):
    """A run stopped after 3 iterations and resumed from its checkpoint ends
    with mcl_run's iterations and clusters."""
    from paper_2002_10083_gb300 import checkpoint
    A = synth.config("planted2k", seed=3).with_val32()
    prm = _prm(theta=1e-4, K=100, p=0.9, iters=30)
    lab0, it0, hist0, _, nc0 = ctx.run(_dev(A), prm, keep_final=False)
    path = str(tmp_path / "run.npz")
    lab1, it1, _, _, _ = checkpoint.run(ctx, A, prm, path, stop_after=3)
    assert lab1 is None and it1 == 3
    lab2, it2, hist2, _, conv2 = checkpoint.run(ctx, A, prm, path)
    assert conv2 == (not nc0) and it2 == it0
    assert np.array_equal(lab2.cpu().numpy(), lab0.cpu().numpy())
    # runs are bit-identical: the resumed history equals the uninterrupted one
    assert list(hist2) == list(hist0)
