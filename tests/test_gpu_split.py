"""GPU tests of the split expansion with the binary merge (Section IV,
Algorithm 2), through the C ABI.

The partial products carry the numeric pass's exact fixed-point sums, so the
merged and pruned iteration must equal mcl_expand bit for bit, for every
stage count; the merge schedule's sizes must equal the oracle's
(oracle/merge.py) exactly, and the iteration must match the FP64 oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2002_10083_gb300 import synth
from tests.parity import compare_iteration

torch = pytest.importorskip("torch")
pytest.importorskip("scipy")
from oracle import merge  # noqa: E402

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


def _prm(theta=1e-4, K=100, p=0.9, Krec=0, r=2.0):
    from paper_2002_10083_gb300 import mcl
    return mcl.Params(threshold=theta, select_k=K, recover_pct=p, recover_k=Krec, inflation=r,
                      chaos_eps=1e-3, max_iters=30)


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


def _merge_stats_equal(st, want):
    for f in ("stages", "merges", "partial_entries", "binary_peak_entries",
              "live_peak_entries", "merged_entries"):
        assert st[f] == getattr(want, f), (f, st[f], getattr(want, f))


@pytest.mark.parametrize("n,dens,seed", [(300, 0.03, 0), (1000, 0.01, 1), (2777, 0.004, 2)])
@pytest.mark.parametrize("ns", [1, 2, 3, 4, 5, 8, 13])
def test_split_equals_one_pass_and_schedule(ctx, n, dens, seed, ns):
    A = synth.random_sparse(n, dens, seed=seed, w="lognormal").with_val32()
    prm = _prm()
    D = _dev(A)
    ref, ch_ref = ctx.expand(D, prm)
    out, ch, st = ctx.expand_split(D, prm, ns)
    torch.cuda.synchronize()
    _assert_same(out, ref)
    assert ch == ch_ref
    _merge_stats_equal(st, merge.binary_merge(A, ns))


@pytest.mark.parametrize("K,p,theta,r", [(20, 0.5, 1e-3, 2.0), (4096, 1.0, 0.0, 1.5),
                                         (1, 0.9, 1e-4, 3.0)])
def test_split_matches_oracle(ctx, K, p, theta, r):
    A = synth.random_sparse(1500, 0.008, seed=7, w="lognormal").with_val32()
    prm = _prm(theta=theta, K=K, p=p, r=r)
    out, ch, _ = ctx.expand_split(_dev(A), prm, 6)
    torch.cuda.synchronize()
    rep, res = compare_iteration(A, out.to_host(), _oprm(prm), rtol=RTOL)
    assert rep.ok(), rep.failures[:5]
    assert abs(ch - float(res.chaos.max())) <= 3 * RTOL * max(1.0, float(res.chaos.max()))


def test_split_power_law_memory(ctx):
    """A power-law graph (Chung-Lu, mean degree 50): bit-identical to the
    one-pass iteration, the schedule equal to the oracle's, and the binary
    merge's largest merge smaller than what a multiway merge holds."""
    A = synth.chung_lu(n=10000, mean=50.0, d_max=1000, seed=3).with_val32()
    prm = _prm(K=1100)
    D = _dev(A)
    ref, _ = ctx.expand(D, prm)
    for ns in (8, 16):
        out, _, st = ctx.expand_split(D, prm, ns)
        torch.cuda.synchronize()
        _assert_same(out, ref)
        _merge_stats_equal(st, merge.binary_merge(A, ns))
        assert st["merged_entries"] < st["binary_peak_entries"] < st["partial_entries"]


def test_split_edge_cases(ctx):
    from paper_2002_10083_gb300 import mcl
    prm = _prm()
    # empty matrix
    E = synth.CSC(n=0, colptr=np.zeros(1, np.int64), rowidx=np.zeros(0, np.int32), val=np.zeros(0))
    out, ch, st = ctx.expand_split(_dev(E), prm, 4)
    assert out.n == 0 and out.nnz == 0 and ch == 0.0 and st["merged_entries"] == 0
    # empty columns, more stages than rows
    A = synth.random_csc(40, 40, 0.2, seed=3, lo=0.1, hi=1.0, empty_cols=(0, 5, 39)).with_val32()
    D = _dev(A)
    ref, _ = ctx.expand(D, prm)
    for ns in (40, 64, 1):
        out, _, st = ctx.expand_split(D, prm, ns)
        torch.cuda.synchronize()
        _assert_same(out, ref)
        _merge_stats_equal(st, merge.binary_merge(A, ns))
    for bad in (0, -1, 4097):
        with pytest.raises(mcl.MclError):
            ctx.expand_split(D, prm, bad)
