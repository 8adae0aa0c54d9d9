"""Pins of the Cohen-estimator oracle (oracle/cohen.py): the splitmix64
generator against its published first outputs, the exact one-vertex case,
the estimator's expectation (the reach size) over many seeds, and the
paper's accuracy claim on an aggregate."""
import numpy as np
import pytest

import oracle
from oracle import cohen
from paper_2002_10083_gb300 import synth


def test_splitmix64_published_sequence():
    # SplittableRandom / splitmix64 from state 0: the first outputs are
    # 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F
    outs = []
    state = np.uint64(0)
    for _ in range(3):
        outs.append(int(cohen.splitmix64(np.array([state]))[0]))
        with np.errstate(over="ignore"):
            state = np.uint64(state + cohen.GOLDEN)
    assert outs == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_keys_are_exponential():
    K = cohen.keys(20000, 5, seed=7)
    assert (K > 0).all()
    # Exp(1): mean 1, variance 1, P(X > 1) = e^-1
    assert abs(K.mean() - 1.0) < 0.02
    assert abs(K.var() - 1.0) < 0.05
    assert abs((K > 1.0).mean() - np.exp(-1.0)) < 0.01


def _single_reach(n_rows_reached, n=None):
    """Column 0 reaches exactly rows 0..N-1 through one middle vertex."""
    N = n_rows_reached
    n = n or N + 1
    # column 0 = {N}; column N = rows {0..N-1}; other columns empty
    colptr = np.zeros(n + 1, np.int64)
    rows = []
    for j in range(n):
        if j == 0:
            rows.append([N])
        elif j == N:
            rows.append(list(range(N)))
        else:
            rows.append([])
        colptr[j + 1] = colptr[j] + len(rows[-1])
    return synth.CSC(n=n, colptr=colptr, rowidx=np.array(sum(rows, []), np.int32),
                     val=np.ones(int(colptr[-1])))


def test_one_reached_row_is_exact_formula():
    A = _single_reach(1)
    r, seed = 6, 11
    est = cohen.estimate(A, r, seed)
    K = cohen.keys(A.n, r, seed)
    assert est[0] == pytest.approx((r - 1) / K[0].sum(), rel=1e-15)


@pytest.mark.parametrize("N,r", [(50, 8), (400, 5)])
def test_estimate_is_unbiased_for_the_reach_size(N, r):
    # sum of the r minima ~ Gamma(r, N) => E[(r-1)/S] = N, sd = N / sqrt(r-2)
    A = _single_reach(N)
    ests = np.array([cohen.estimate(A, r, seed)[0] for seed in range(300)])
    sd_mean = N / np.sqrt(r - 2) / np.sqrt(len(ests))
    assert abs(ests.mean() - N) < 4 * sd_mean


@pytest.mark.parametrize("r", [3, 5, 7, 10])
def test_aggregate_within_ten_percent(r):
    # Section VII-C: a few keys estimate the memory requirement within ~10%
    A = synth.random_sparse(3000, 0.004, seed=5)
    _, exact = oracle.symbolic_cols(A)
    est = cohen.estimate(A, r, seed=2002)
    assert abs(est.sum() / exact.sum() - 1.0) < 0.10
