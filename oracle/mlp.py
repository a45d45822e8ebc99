"""FP64 oracle of the learned alpha proposal: features, the MLP, its loss,
analytic gradients and the Adam update.

TEST INFRASTRUCTURE, like the rest of this package: only the test suite,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it; the CUDA library never does, and this module imports nothing from it.

The paper computes alpha as the root of Eq. (entropic) and has no learned
part; the proposal is an addition: a small network guesses the root, and a
Newton correction on the paper's h(alpha) (with the plain Newton root as the
fallback) keeps the result the method's root. What this module fixes:

* features of a site (populations f_p, Delta_p = f^eq_p - f_p): with
  x_p = Delta_p / f_p and S = max_p |x_p|,
  X = (x_0/S, ..., x_18/S, (log2 S + 9)/8);
* the network o(X) = W3 . gelu(W2 gelu(W1 X + b1) + b2) + b3, 20 -> 64 ->
  64 -> 1, gelu the tanh form of Hendrycks & Gimpel (2016),
  gelu(z) = z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3)));
* the moment-series start alpha_c: the root of the cubic truncation
  h(a)/a ~ h'(0) + a M2/2 - a^2 M3/6 + a^3 M4/12 (M_k = sum_p f_p x_p^k; the
  expansion of phi(a x) = (a x)^2/2 - (a x)^3/6 + (a x)^4/12 - ...), reached by
  three Newton steps from -2 h'(0)/M2 (a step is kept only inside (0, 8));
  its error is O(S^3);
* the proposal alpha = alpha_c + S^3 o(X) where S >= 2^-5 (below, the
  correction is under the FP32 resolution of alpha_c and the proposal is
  alpha_c), so the regression target of a site with root alpha* is
  o* = (alpha* - alpha_c)/S^3;
* loss = mean over the batch of (o - o*)^2;
* Adam (Kingma & Ba 2015, Algorithm 1) with bias correction.

Parameters are one flat FP64 vector in the order W1 (64 x 20, row-major:
out x in), b1 (64), W2 (64 x 64), b2 (64), W3 (64), b3 (1); 5569 values.
"""
from __future__ import annotations

import math

import numpy as np

NIN, NH = 20, 64
SHAPES = [("W1", (NH, NIN)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("W3", (NH,)), ("b3", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)
_C = math.sqrt(2.0 / math.pi)
_K = 0.044715


def unpack(theta):
    out, k = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = theta[k:k + n].reshape(shape)
        k += n
    return out


def pack(parts):
    return np.concatenate([np.asarray(parts[name], np.float64).reshape(-1) for name, _ in SHAPES])


def init_params(seed):
    """Glorot-uniform weights (Glorot & Bengio 2010), zero biases."""
    rng = np.random.default_rng(seed)
    parts = {}
    for name, shape in SHAPES:
        if name.startswith("W"):
            fan_out, fan_in = (shape[0], shape[1]) if len(shape) == 2 else (1, shape[0])
            lim = math.sqrt(6.0 / (fan_in + fan_out))
            parts[name] = rng.uniform(-lim, lim, size=shape)
        else:
            parts[name] = np.zeros(shape)
    return pack(parts)


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(_C * (z + _K * z ** 3)))


def gelu_prime(z):
    t = np.tanh(_C * (z + _K * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * _C * (1.0 + 3.0 * _K * z * z)


def features(f, delta):
    """X (n, 20) and S (n,) from populations f (19, n) and Delta (19, n)."""
    x = delta / f
    S = np.max(np.abs(x), axis=0)
    S = np.where(S > 0, S, 1.0)
    X = np.empty((f.shape[1], NIN))
    X[:, :19] = (x / S).T
    X[:, 19] = (np.log2(S) + 9.0) / 8.0
    return X, S


def forward(theta, X):
    """o (n,) and the intermediates of the pass."""
    P = unpack(theta)
    z1 = X @ P["W1"].T + P["b1"]
    h1 = gelu(z1)
    z2 = h1 @ P["W2"].T + P["b2"]
    h2 = gelu(z2)
    o = h2 @ P["W3"] + P["b3"][0]
    return o, (z1, h1, z2, h2)


def loss(theta, X, y):
    o, _ = forward(theta, X)
    return float(np.mean((o - y) ** 2))


def grad(theta, X, y):
    """Analytic gradient of the mean squared error (back-propagation through
    the three affine maps and two gelu layers)."""
    P = unpack(theta)
    o, (z1, h1, z2, h2) = forward(theta, X)
    n = X.shape[0]
    do = 2.0 * (o - y) / n                 # (n,)
    g = {"W3": h2.T @ do, "b3": np.array([do.sum()])}
    dz2 = np.outer(do, P["W3"]) * gelu_prime(z2)   # (n, 64)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ P["W2"]) * gelu_prime(z1)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(axis=0)
    return pack(g), float(np.mean((o - y) ** 2))


def adam(theta, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (t counts from 1); returns the new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def series_start(f, delta, h0):
    """alpha_c of each site (f, Delta (19, n); h0 = h'(0) (n,))."""
    x = delta / f
    M2 = np.sum(f * x ** 2, axis=0)
    M3 = np.sum(f * x ** 3, axis=0)
    M4 = np.sum(f * x ** 4, axis=0)
    a = -2.0 * h0 / M2
    for _ in range(3):
        g = h0 + a * (0.5 * M2 + a * (-M3 / 6.0 + a * (M4 / 12.0)))
        gp = 0.5 * M2 + a * (-M3 / 3.0 + a * (M4 / 4.0))
        an = a - g / gp
        a = np.where((an > 0) & (an < 8), an, a)
    return a


S_MIN = 2.0 ** -5


def proposal(theta, f, delta, h0):
    """alpha proposed for each site: alpha_c + S^3 o(X) where S >= S_MIN."""
    X, S = features(f, delta)
    o, _ = forward(theta, X)
    return series_start(f, delta, h0) + np.where(S >= S_MIN, S ** 3 * o, 0.0)


def target(f, delta, h0, alpha_root):
    """Regression target o* = (alpha* - alpha_c)/S^3."""
    _, S = features(f, delta)
    return (alpha_root - series_start(f, delta, h0)) / S ** 3
