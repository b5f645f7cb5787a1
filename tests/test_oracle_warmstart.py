"""Pins of the warm-start oracle (oracle/warmstart.py) to facts that do not
come from the oracle itself: order statistics of columns built with known
sorted values, counts of a planted utility mix, the textbook value of GELU
and its odd-part identity, a network whose weights reduce it to a scalar
closed form, invariance under relabelling hidden units (catches a transposed
or mis-indexed weight), central finite differences of the loss (pins the
back-propagation), and Adam's closed form under a constant gradient."""
import math

import numpy as np
import pytest

from oracle import warmstart as WS


def test_quantiles_of_a_permuted_column_small_n():
    n, m = 1000, 3
    rng = np.random.default_rng(0)
    scale = np.array([0.5, 2.0, 7.0])
    A = np.empty((n, m))
    for j in range(m):
        A[:, j] = (rng.permutation(n) + 1) * scale[j]
    st = WS.resource_stats(A, np.zeros(n, np.uint8), np.ones(n), np.full(m, 10.0))
    for j in range(m):
        for l in range(8):
            k = ((2 * l + 1) * n) // 16          # 0-based order statistic
            assert st[j, l] == pytest.approx(math.log((k + 1) * scale[j]), abs=1e-15)
        assert st[j, 8] == pytest.approx(math.log(10.0 / n), abs=1e-15)


def test_quantiles_use_the_strided_sample_above_16384_rows():
    n = 50_000
    A = np.arange(n, dtype=np.float64)[:, None] + 1.0     # A_i = i + 1, increasing
    st = WS.resource_stats(A, np.zeros(n, np.uint8), np.ones(n), np.array([1.0]))
    S = 16384
    for l in range(8):
        k = ((2 * l + 1) * S) // 16
        row = (k * n) // S                                  # k-th sampled row
        assert st[0, l] == pytest.approx(math.log(row + 1.0), abs=1e-15)


def test_utility_fractions_and_mean_log_weight():
    n = 800
    kind = np.array([0] * 400 + [1] * 200 + [2] * 120 + [3] * 80, np.uint8)
    w = np.where(np.arange(n) % 2 == 0, 1.0, math.e ** 2)   # log w alternates 0, 2
    st = WS.resource_stats(np.ones((n, 2)), kind, w, np.ones(2))
    assert np.allclose(st[:, 9], 0.5) and np.allclose(st[:, 10], 0.25)
    assert np.allclose(st[:, 11], 0.25) and np.allclose(st[:, 12], 1.0)
    X = WS.features(np.ones((n, 2)), kind, w, np.array([1.0, 3.0]))
    assert X.shape == (2, 26)
    assert X[0, 13 + 8] == pytest.approx(0.5 * (math.log(1 / n) + math.log(3 / n)))


def test_gelu_textbook_values():
    # GELU(x) = x Phi(x); Phi(1) = 0.841344746068543, Phi(3) = 0.998650101968370
    assert WS.gelu(np.array([0.0]))[0] == 0.0
    assert WS.gelu(np.array([1.0]))[0] == pytest.approx(0.841344746068543, rel=1e-14)
    assert WS.gelu(np.array([3.0]))[0] == pytest.approx(3 * 0.998650101968370, rel=1e-14)
    x = np.linspace(-4, 4, 33)
    assert np.allclose(WS.gelu(x) - WS.gelu(-x), x, atol=1e-15)   # x Phi(x) + x Phi(-x) = x
    h = 1e-6
    fd = (WS.gelu(x + h) - WS.gelu(x - h)) / (2 * h)
    assert np.allclose(WS.gelu_grad(x), fd, atol=1e-8)


def test_forward_reduces_to_a_scalar_closed_form():
    # W1 routes input 0 to hidden unit 0, W2 is the identity, W3 picks unit 0:
    # y = GELU(GELU(x_0 + b)) + c
    P = {name: np.zeros(shape) for name, shape in WS.SHAPES}
    P["W1"][0, 0] = 1.0
    P["b1"][0] = 0.25
    P["W2"] = np.eye(WS.HIDDEN)
    P["W3"][0] = 1.0
    P["b3"][0] = -0.5
    X = np.random.default_rng(1).normal(size=(5, 26))
    y = WS.forward(WS.pack(P), X)
    Phi = lambda z: 0.5 * (1 + math.erf(z / math.sqrt(2)))
    for r in range(5):
        z = X[r, 0] + 0.25
        g1 = z * Phi(z)
        assert y[r] == pytest.approx(g1 * Phi(g1) - 0.5, rel=1e-13, abs=1e-15)


def test_forward_is_invariant_under_relabelling_hidden_units():
    rng = np.random.default_rng(2)
    theta = rng.normal(scale=0.2, size=WS.N_PARAMS)
    P = WS.unpack(theta)
    X = rng.normal(size=(7, 26))
    p1, p2 = rng.permutation(WS.HIDDEN), rng.permutation(WS.HIDDEN)
    Q = {"W1": P["W1"][:, p1], "b1": P["b1"][p1], "W2": P["W2"][p1][:, p2], "b2": P["b2"][p2],
         "W3": P["W3"][p2], "b3": P["b3"]}
    assert np.allclose(WS.forward(theta, X), WS.forward(WS.pack(Q), X), rtol=1e-12, atol=1e-12)


def test_gradients_match_central_differences():
    rng = np.random.default_rng(3)
    theta = rng.normal(scale=0.15, size=WS.N_PARAMS)
    X = rng.normal(size=(6, 26))
    t = rng.normal(size=6)
    L, g = WS.loss_and_grads(theta, X, t)
    assert L == pytest.approx(np.mean((WS.forward(theta, X) - t) ** 2), rel=1e-14)
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in WS.SHAPES])
    picks = []
    for a, b in zip(offs[:-1], offs[1:]):       # a few coordinates of every tensor
        picks += list(rng.choice(np.arange(a, b), size=min(6, b - a), replace=False))
    h = 1e-6
    for i in picks:
        e = np.zeros_like(theta)
        e[i] = h
        fd = (WS.loss_and_grads(theta + e, X, t)[0] - WS.loss_and_grads(theta - e, X, t)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-9), i


def test_adam_constant_gradient_closed_form():
    # with a constant gradient g, mhat = g and vhat = g^2 at every step, so each
    # step moves theta by lr g / (|g| + eps)
    g = np.array([2.0, -0.5, 1e-3, -7.0])
    theta, m, v = np.zeros(4), np.zeros(4), np.zeros(4)
    lr = 0.01
    for t in range(1, 6):
        theta, m, v = WS.adam(theta, g, m, v, t, lr)
        assert np.allclose(theta, -t * lr * g / (np.abs(g) + WS.ADAM_EPS), rtol=1e-12, atol=1e-15)


def test_training_with_the_oracle_reduces_the_loss():
    rng = np.random.default_rng(4)
    X = rng.normal(size=(64, 26))
    t = np.tanh(X[:, 0]) - 0.5 * X[:, 3]
    theta = rng.normal(scale=0.05, size=WS.N_PARAMS)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    L0 = WS.loss_and_grads(theta, X, t)[0]
    for step in range(1, 61):
        L, g = WS.loss_and_grads(theta, X, t)
        theta, m, v = WS.adam(theta, g, m, v, step, 3e-3)
    assert WS.loss_and_grads(theta, X, t)[0] < 0.2 * L0
