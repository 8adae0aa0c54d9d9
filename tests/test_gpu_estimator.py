"""GPU tests of the learned output-size estimator through the C ABI:
features, MLP forward and backward against the FP64 oracle (same BF16
weights), one Adam step, a short training run on exact symbolic labels,
and the learned sizing path in mcl_expand (results still match the oracle).
"""
import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
from paper_2002_10083_gb300 import synth
from tests.parity import compare_iteration

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def _weights(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    bits = omlp.bf16_round_bits(rng.normal(0, scale, omlp.NPARAM).astype(np.float32))
    return bits, omlp.bf16_bits_to_f64(bits)


@pytest.mark.parametrize("it,prev", [(1, False), (3, True)])
def test_features_match_oracle(ctx, it, prev):
    A = synth.chung_lu(n=5000, mean=20.0, d_max=1500, seed=3).with_val32()
    D = _dev(A)
    pl = None
    if prev:
        pl = np.random.default_rng(0).normal(0, 1, A.n).astype(np.float32)
    F = ctx.features(D, it, torch.from_numpy(pl).cuda() if prev else None).cpu().numpy()
    O = omlp.column_features(A, iteration=it, prev_logcf=pl)
    np.testing.assert_allclose(F, O, rtol=2e-6, atol=2e-6)


def test_forward_matches_oracle(ctx):
    bits, theta = _weights(1)
    rng = np.random.default_rng(2)
    X = rng.normal(0, 2, (3000, omlp.NIN)).astype(np.float32)
    mu = rng.normal(0, 0.5, omlp.NIN).astype(np.float32)
    sg = rng.uniform(0.5, 2, omlp.NIN).astype(np.float32)
    norm = np.concatenate([mu, sg])
    w = torch.from_numpy(bits.view(np.int16)).cuda()
    Y = ctx.mlp_forward(torch.from_numpy(X).cuda(), w, torch.from_numpy(norm).cuda()).cpu().numpy()
    Yo = omlp.forward(theta, X.astype(np.float64), mu.astype(np.float64), sg.astype(np.float64))
    np.testing.assert_allclose(Y, Yo, rtol=1e-4, atol=1e-4)


def test_backward_matches_oracle(ctx):
    bits, theta = _weights(4, 0.2)
    rng = np.random.default_rng(5)
    B = 777
    X = rng.normal(0, 1, (B, omlp.NIN)).astype(np.float32)
    T = rng.normal(0, 1, (B, omlp.NOUT)).astype(np.float32)
    norm = np.concatenate([np.zeros(omlp.NIN), np.ones(omlp.NIN)]).astype(np.float32)
    w = torch.from_numpy(bits.view(np.int16)).cuda()
    grad = torch.zeros(omlp.NPARAM, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.mlp_backward(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda(), w,
                     torch.from_numpy(norm).cuda(), 1.0 / B, grad, loss)
    Lo, go = omlp.grad(theta, X.astype(np.float64), T.astype(np.float64), np.zeros(omlp.NIN),
                       np.ones(omlp.NIN))
    g = grad.cpu().numpy().astype(np.float64)
    assert abs(loss.item() / B - Lo) <= 1e-5 * Lo
    assert np.linalg.norm(g - go) <= 1e-3 * np.linalg.norm(go)
    big = np.abs(go) > 1e-3 * np.abs(go).max()
    np.testing.assert_allclose(g[big], go[big], rtol=1e-3, atol=1e-5 * np.abs(go).max())


def test_adam_step(ctx):
    rng = np.random.default_rng(6)
    master = rng.normal(0, 0.1, omlp.NPARAM).astype(np.float32)
    m = rng.normal(0, 0.01, omlp.NPARAM).astype(np.float32)
    v = rng.uniform(0, 0.01, omlp.NPARAM).astype(np.float32)
    g = rng.normal(0, 0.1, omlp.NPARAM).astype(np.float32)
    t = [torch.from_numpy(x.copy()).cuda() for x in (master, m, v, g)]
    wb = torch.zeros(omlp.NPARAM, dtype=torch.int16, device="cuda")
    ctx.adam_step(t[0], t[1], t[2], t[3], 3, 1e-2, wb)
    b1, b2, eps = 0.9, 0.999, 1e-8
    m2 = b1 * m.astype(np.float64) + (1 - b1) * g
    v2 = b2 * v.astype(np.float64) + (1 - b2) * g.astype(np.float64) ** 2
    w2 = master - 1e-2 * (m2 / (1 - b1 ** 3)) / (np.sqrt(v2 / (1 - b2 ** 3)) + eps)
    np.testing.assert_allclose(t[0].cpu().numpy(), w2, rtol=1e-5, atol=1e-7)
    np.testing.assert_array_equal(wb.cpu().numpy().view(np.uint16),
                                  omlp.bf16_round_bits(t[0].cpu().numpy()))


@pytest.fixture(scope="module")
def trained(ctx):
    from paper_2002_10083_gb300 import estimator
    A = synth.chung_lu(n=30000, mean=40.0, d_max=3000, seed=11).with_val32()
    X, T = estimator.collect(ctx, A, iterations=2, sample=0)
    wb, norm, hist = estimator.train(ctx, X, T, epochs=12, batch=2048, lr=3e-3)
    return A, X, T, wb, norm, hist


def test_training_reduces_loss(trained, ctx):
    from paper_2002_10083_gb300 import estimator
    A, X, T, wb, norm, hist = trained
    assert hist[-1] < 0.5 * hist[0], hist
    stats, ratio = estimator.evaluate(ctx, X, T, wb, norm)
    # a short run already predicts nnz within a factor of ~1.5 for most columns
    assert stats["median_abs_log_ratio"] < 0.4, stats


def test_learned_sizing_same_results(trained, ctx):
    from paper_2002_10083_gb300 import mcl
    A, X, T, wb, norm, hist = trained
    ctx.estimator_load(wb.cpu().numpy().view(np.uint16), norm.cpu().numpy(), 1.2)
    prm = mcl.Params(threshold=1e-4, select_k=300, recover_pct=0.9, use_estimator=1)
    D = _dev(A)
    est = ctx.estimate(D)
    assert est.min().item() >= 1
    out, ch = ctx.expand(D, prm)
    G = out.to_host()
    cols = np.random.default_rng(3).choice(A.n, 800, replace=False).astype(np.int32)
    oprm = oracle.Params(theta=float(np.float32(1e-4)), K=300, p=float(np.float32(0.9)), r=2.0)
    rep, _ = compare_iteration(A, G, oprm, cols=cols, rtol=1e-5)
    assert rep.ok(), rep.failures[:5]
    # the exact symbolic counts judge the estimate
    fl, nz = ctx.symbolic(D)
    ratio = (nz.double().clamp(min=1) / est.double()).cpu().numpy()
    assert np.median(np.abs(np.log(ratio))) < 0.5
    # the full loop with the estimator matches the plain loop's clusters
    prm_plain = mcl.Params(threshold=1e-4, select_k=300, recover_pct=0.9, max_iters=8)
    prm_learn = mcl.Params(threshold=1e-4, select_k=300, recover_pct=0.9, max_iters=8,
                           use_estimator=1)
    lab_p, it_p, h_p, _, _ = ctx.run(_dev(A), prm_plain, keep_final=False)
    lab_l, it_l, h_l, _, _ = ctx.run(_dev(A), prm_learn, keep_final=False)
    assert it_p == it_l
    # the estimate only plans the windows: bit-identical iterations
    assert h_l == h_p
    assert np.array_equal(lab_l.cpu().numpy(), lab_p.cpu().numpy())


def _prediction(ctx, D):
    """The committed network's prediction of nnz((AA)_*j): expm1 of its
    first output on the first iteration's features (before the safety factor
    and the clamp to the flops and row-span bounds that sizing applies)."""
    from paper_2002_10083_gb300 import estimator
    w, norm, _, _ = estimator.load()
    X = ctx.features(D, 1)
    Y = ctx.mlp_forward(X, torch.from_numpy(w.view(np.int16)).cuda(),
                        torch.from_numpy(norm).cuda())
    return torch.expm1(Y[:, 0].double())


def _median_abs_log_ratio(ctx, D):
    pred = _prediction(ctx, D)
    fl, nz = ctx.symbolic(D)
    ratio = (nz.double().clamp(min=1) / pred.clamp(min=1)).cpu().numpy()
    return float(np.median(np.abs(np.log(ratio))))


def _learned_vs_plain(ctx, D, K=1100):
    """Median time of 3 expansions in each form; the outputs."""
    import time
    from paper_2002_10083_gb300 import mcl
    times, outs = {}, {}
    for name, ue in (("plain", 0), ("learned", 1)):
        prm = mcl.Params(threshold=1e-4, select_k=K, recover_pct=0.9, use_estimator=ue)
        out, ch = ctx.expand(D, prm)  # warm
        del out
        torch.cuda.synchronize()
        t = []
        for _ in range(3):
            t0 = time.perf_counter()
            out, ch = ctx.expand(D, prm)
            torch.cuda.synchronize()
            t.append(time.perf_counter() - t0)
        times[name] = sorted(t)[1]
        outs[name] = (out, ch)
    return times, outs


@pytest.mark.slow
@pytest.mark.parametrize("n", [400_000, 200_000])
def test_trained_estimator_off_the_bench_size(ctx, n):
    """The committed estimator on power-law graphs of 400k and 200k vertices
    (a seed it never saw): predictions within a few percent of the exact
    symbolic counts, and the learned form faster than the plain one."""
    from paper_2002_10083_gb300 import estimator
    estimator.install(ctx)
    A = synth.config("zipf1m", n=n, seed=102).with_val32()
    D = _dev(A)
    assert _median_abs_log_ratio(ctx, D) < 0.05
    times, outs = _learned_vs_plain(ctx, D)
    assert times["learned"] < times["plain"], times
    L, Pn = outs["learned"][0], outs["plain"][0]
    assert torch.equal(L.val.view(torch.int32), Pn.val.view(torch.int32))


def test_trained_estimator_on_a_held_out_batch(ctx):
    """The same network on the planted-partition batch family at a size it
    was not trained on (128 components; trained on 64, 256 and 1024) and a
    seed it never saw: predictions within a few percent, the same iteration
    as the plain form."""
    from paper_2002_10083_gb300 import estimator, mcl
    estimator.install(ctx)
    A = synth.config("batch4096", ncomp=128, seed=102).with_val32()
    D = _dev(A)
    assert _median_abs_log_ratio(ctx, D) < 0.05
    outs = {}
    for ue in (0, 1):
        prm = mcl.Params(threshold=1e-4, select_k=1100, recover_pct=0.9, use_estimator=ue)
        outs[ue] = ctx.expand(D, prm)[0]
    assert torch.equal(outs[0].rowidx, outs[1].rowidx)
    assert torch.equal(outs[0].val.view(torch.int32), outs[1].val.view(torch.int32))


@pytest.mark.slow
def test_trained_estimator_gain_on_held_out_graph(ctx):
    """The committed estimator on the held-out 1M-vertex graph seed 100: its
    estimates are within a few percent of the exact symbolic counts, the
    learned form replaces the symbolic pass and is faster than the plain
    form, and its results match the oracle."""
    import time
    from paper_2002_10083_gb300 import estimator, mcl
    meta = estimator.install(ctx)
    A = synth.config("zipf1m", seed=100).with_val32()
    D = _dev(A)
    est = ctx.estimate(D)
    fl, nz = ctx.symbolic(D)
    ratio = (nz.double().clamp(min=1) / est.double()).cpu().numpy()
    # the prediction within a few percent; the sizing estimate (prediction x
    # safety, clamped to the flops and row-span bounds) covers 95% of the columns
    assert _median_abs_log_ratio(ctx, D) < 0.05
    assert np.quantile(ratio, 0.95) < 1.0
    times = {}
    outs = {}
    for name, ue in (("plain", 0), ("learned", 1)):
        prm = mcl.Params(threshold=1e-4, select_k=1100, recover_pct=0.9, use_estimator=ue)
        out, ch = ctx.expand(D, prm)  # warm
        del out
        torch.cuda.synchronize()
        t = []
        for _ in range(3):
            t0 = time.perf_counter()
            out, ch = ctx.expand(D, prm)
            torch.cuda.synchronize()
            t.append(time.perf_counter() - t0)
        times[name] = sorted(t)[1]
        outs[name] = (out, ch)
    assert times["learned"] < times["plain"], times
    # the same iteration either way, bit for bit
    L, Pn = outs["learned"][0], outs["plain"][0]
    assert torch.equal(L.colptr, Pn.colptr) and torch.equal(L.rowidx, Pn.rowidx)
    assert torch.equal(L.val.view(torch.int32), Pn.val.view(torch.int32))
    assert outs["learned"][1] == outs["plain"][1]
    G = outs["learned"][0].to_host()
    cols = np.random.default_rng(7).choice(A.n, 400, replace=False).astype(np.int32)
    oprm = oracle.Params(theta=float(np.float32(1e-4)), K=1100, p=float(np.float32(0.9)), r=2.0)
    rep, _ = compare_iteration(A, G, oprm, cols=cols, rtol=1e-5)
    assert rep.ok(), rep.failures[:5]
