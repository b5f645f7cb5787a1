"""FP64 CPU oracle of the learned warm start (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module; it imports nothing from the product
package.  Plain numpy in FP64, written to be checked by eye:

* ``features``     per-resource summary statistics of a problem (13 numbers
                   per resource) and the network input (26 = those 13 plus
                   their mean over the problem's resources)
* ``forward``      the shared per-resource MLP 26 -> 256 -> 256 -> 1 with
                   GELU (Hendrycks and Gimpel 2016, exact erf form); the
                   output is log(lambda_j)
* ``loss_and_grads``  mean squared error on log(lambda*) and its gradient by
                   back-propagation through the three layers
* ``adam``         one Adam update (Kingma and Ba 2015, Algorithm 1)

The cold start these prices compete with is Eq. e-initialization of the
paper (``oracle.init_prices``); the rule that keeps the cold start when the
learned prices give a larger dual value g is the fallback of the warm start.

Parameter layout (one flat vector, also the library's): W1 (26 x 256,
row-major, input-major), b1 (256), W2 (256 x 256), b2 (256), W3 (256), b3 (1).
"""
from __future__ import annotations

import math

import numpy as np

F_RES = 13               # statistics per resource
F_IN = 2 * F_RES         # network input per resource
HIDDEN = 256
N_QUANT = 8
SAMPLE_MAX = 16384
SHAPES = [("W1", (F_IN, HIDDEN)), ("b1", (HIDDEN,)), ("W2", (HIDDEN, HIDDEN)), ("b2", (HIDDEN,)),
          ("W3", (HIDDEN,)), ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)
TINY = 1e-30             # floor inside the logarithms (A_ij may be 0)


def sample_rows(n: int) -> np.ndarray:
    """The rows the statistics are taken over: all rows when n <= 16384,
    else the strided sample i_k = floor(k n / S), k = 0 .. S-1, S = 16384."""
    S = min(n, SAMPLE_MAX)
    return (np.arange(S, dtype=np.int64) * n) // S


def quantile_index(S: int, l: int) -> int:
    """Order statistic used as quantile l of 8: the one at level (2l+1)/16."""
    return ((2 * l + 1) * S) // 16


def resource_stats(A, kind, w, R) -> np.ndarray:
    """(m, 13): for resource j, log of the 8 quantiles of A[:, j] over the
    sample, log(R_j / n), the fractions of log, power and linear (linear with
    cap and target) utilities over the sample, and the mean of log w over
    the sample (the last four are the same for every j)."""
    n, m = A.shape
    rows = sample_rows(n)
    S = len(rows)
    As = np.asarray(A, dtype=np.float64)[rows]
    ks = np.asarray(kind)[rows]
    ws = np.asarray(w, dtype=np.float64)[rows]
    out = np.zeros((m, F_RES))
    for j in range(m):
        col = np.sort(As[:, j])
        for l in range(N_QUANT):
            out[j, l] = math.log(max(col[quantile_index(S, l)], TINY))
        out[j, 8] = math.log(max(float(R[j]) / n, TINY))
    out[:, 9] = np.count_nonzero(ks == 0) / S
    out[:, 10] = np.count_nonzero(ks == 1) / S
    out[:, 11] = np.count_nonzero(ks >= 2) / S
    out[:, 12] = float(np.mean(np.log(np.maximum(ws, TINY))))
    return out


def features(A, kind, w, R) -> np.ndarray:
    """(m, 26) network input: each resource's 13 statistics followed by the
    mean of those statistics over the problem's m resources."""
    st = resource_stats(A, kind, w, R)
    return np.concatenate([st, np.repeat(st.mean(0, keepdims=True), st.shape[0], 0)], axis=1)


def unpack(theta: np.ndarray) -> dict:
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.size == N_PARAMS
    out, pos = {}, 0
    for name, shape in SHAPES:
        size = int(np.prod(shape))
        out[name] = theta[pos:pos + size].reshape(shape)
        pos += size
    return out


def pack(parts: dict) -> np.ndarray:
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def gelu(z):
    """GELU(z) = z Phi(z), Phi the standard normal CDF, Phi(z) = (1 + erf(z / sqrt 2)) / 2."""
    from scipy.special import erf
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    """d/dz [z Phi(z)] = Phi(z) + z phi(z), phi the standard normal density."""
    from scipy.special import erf
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(theta, X, keep=False):
    """y = W3 . GELU(GELU(X W1 + b1) W2 + b2) + b3 for each row of X (rows x 26)."""
    P = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ P["W1"] + P["b1"]
    h1 = gelu(z1)
    z2 = h1 @ P["W2"] + P["b2"]
    h2 = gelu(z2)
    y = h2 @ P["W3"] + P["b3"][0]
    if keep:
        return y, dict(X=X, z1=z1, h1=h1, z2=z2, h2=h2)
    return y


def loss_and_grads(theta, X, target):
    """L = (1/rows) sum_r (y_r - target_r)^2 and dL/dtheta (flat, the
    parameter layout) by the chain rule through the three layers."""
    P = unpack(theta)
    y, c = forward(theta, X, keep=True)
    t = np.asarray(target, dtype=np.float64)
    rows = len(t)
    r = y - t
    L = float(np.mean(r * r))
    dy = 2.0 * r / rows                       # dL/dy
    g = {}
    g["W3"] = c["h2"].T @ dy
    g["b3"] = np.array([dy.sum()])
    dz2 = np.outer(dy, P["W3"]) * gelu_grad(c["z2"])
    g["W2"] = c["h1"].T @ dz2
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ P["W2"].T) * gelu_grad(c["z1"])
    g["W1"] = c["X"].T @ dz1
    g["b1"] = dz1.sum(0)
    return L, pack(g)


ADAM_B1, ADAM_B2, ADAM_EPS = 0.9, 0.999, 1e-8


def adam(theta, grad, m, v, t, lr):
    """One Adam step (Kingma and Ba 2015, Algorithm 1) at step number t >= 1:
    m <- b1 m + (1 - b1) g;  v <- b2 v + (1 - b2) g^2;
    theta <- theta - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
    Returns (theta, m, v)."""
    m = ADAM_B1 * m + (1.0 - ADAM_B1) * grad
    v = ADAM_B2 * v + (1.0 - ADAM_B2) * grad * grad
    mhat = m / (1.0 - ADAM_B1 ** t)
    vhat = v / (1.0 - ADAM_B2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + ADAM_EPS), m, v
