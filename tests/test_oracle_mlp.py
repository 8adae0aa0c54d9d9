"""Pins of the estimator oracle (oracle/mlp.py): gradients against central
finite differences, a hand-built network with a closed-form output, BF16
rounding against torch's conversion, and hand-computed features."""
import numpy as np
import pytest

from oracle import mlp
from paper_2002_10083_gb300 import synth


def _rand_theta(rng, scale=0.3):
    return mlp.bf16_bits_to_f64(mlp.bf16_round_bits(rng.normal(0, scale, mlp.NPARAM)))


@pytest.mark.parametrize("seed", range(3))
def test_gradient_matches_central_differences(seed):
    rng = np.random.default_rng(seed)
    theta = _rand_theta(rng)
    X = rng.normal(0, 1, (7, mlp.NIN))
    T = rng.normal(0, 1, (7, mlp.NOUT))
    mu = rng.normal(0, 0.1, mlp.NIN)
    sg = rng.uniform(0.5, 2.0, mlp.NIN)
    L, g = mlp.grad(theta, X, T, mu, sg)
    assert abs(L - mlp.loss(theta, X, T, mu, sg)) < 1e-12
    idx = rng.choice(mlp.NPARAM, 120, replace=False)
    h = 1e-6
    for p in idx:
        tp = theta.copy(); tp[p] += h
        tm = theta.copy(); tm[p] -= h
        fd = (mlp.loss(tp, X, T, mu, sg) - mlp.loss(tm, X, T, mu, sg)) / (2 * h)
        # ReLU kinks are measure-zero for random inputs
        assert abs(fd - g[p]) <= 1e-6 * max(1.0, abs(fd)), (p, fd, g[p])


def test_hand_built_network():
    P = {name: np.zeros(shp) for name, shp in mlp.SHAPES}
    P["W1"][0, 0] = 1.0
    P["W2"][0, 0] = 2.0
    P["W3"][0, 0] = 3.0
    P["b3"][:] = [0.5, -1.0]
    theta = mlp.pack(P)
    X = np.zeros((3, mlp.NIN))
    X[:, 0] = [2.0, -1.0, 0.25]
    Y = mlp.forward(theta, X, np.zeros(mlp.NIN), np.ones(mlp.NIN))
    np.testing.assert_array_equal(Y[:, 0], [12.5, 0.5, 2.0])
    np.testing.assert_array_equal(Y[:, 1], [-1.0, -1.0, -1.0])
    # standardisation: (x - mu) / sigma
    Y2 = mlp.forward(theta, X, np.full(mlp.NIN, 1.0), np.full(mlp.NIN, 2.0))
    np.testing.assert_array_equal(Y2[:, 0], [6 * 0.5 + 0.5, 0.5, 0.5])


def test_bf16_rounding_against_torch():
    torch = pytest.importorskip("torch")
    x = np.array([1.0, 1.00390625, 1.01171875, -3.14159, 1e-20, 65504.0, 0.1, 2.5e-3],
                 dtype=np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    np.testing.assert_array_equal(mlp.bf16_round_bits(x), want)
    # halfway cases go to even
    assert mlp.bf16_round_bits(np.float32([1.00390625]))[0] == 0x3F80
    assert mlp.bf16_round_bits(np.float32([1.01171875]))[0] == 0x3F82


def test_features_hand_example():
    # path 0 - 1 - 2 with loops (weights 1), column-normalised
    A = synth.assemble(3, np.array([0, 1]), np.array([1, 2]), np.array([1.0, 1.0]), loop="one")
    F = mlp.column_features(A, iteration=2)
    deg = np.diff(A.colptr)
    assert list(deg) == [2, 3, 2]
    # column 1 references columns 0, 1, 2 of sizes 2, 3, 2
    np.testing.assert_allclose(F[1, 0], np.log1p(3))
    np.testing.assert_allclose(F[1, 1], np.log1p(7))
    np.testing.assert_allclose(F[1, 2], np.log1p(3))
    np.testing.assert_allclose(F[1, 3], np.log1p(7 / 3))
    np.testing.assert_allclose(F[1, 4], np.log1p((4 + 9 + 4) / 3 - (7 / 3) ** 2))
    np.testing.assert_allclose(F[1, 5:8], [1 / 3, 1.0, 1 / 3])
    np.testing.assert_allclose(F[1, 8], np.log1p(3))
    assert F[1, 9] == 0.0
    np.testing.assert_allclose(F[1, 10], np.log(3))
    np.testing.assert_allclose(F[1, 11], np.log1p(2))
    assert F[1, 12] == 0.0
    # max values of columns 0, 1, 2 are 1/2, 1/3, 1/2
    np.testing.assert_allclose(F[1, 13], (0.5 + 1 / 3 + 0.5) / 3)
    np.testing.assert_allclose(F[1, 14], np.log1p(3))
    assert F[1, 15] == 1.0
    # column 0 references columns 0, 1 (sizes 2, 3): rows 0..2 reachable
    np.testing.assert_allclose(F[0, 1], np.log1p(5))
    np.testing.assert_allclose(F[0, 14], np.log1p(3))
    np.testing.assert_allclose(F[0, 8], np.log1p(2))
