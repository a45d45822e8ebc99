"""Pins of the learned-alpha oracle (oracle/mlp.py) against things other than
itself: central finite differences, the exact erf form of gelu, the closed
form of Adam's first step, scale invariance of the features."""
import math

import numpy as np

from oracle import mlp


def _batch(n=7, seed=3):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, mlp.NIN))
    y = rng.normal(size=n)
    theta = mlp.init_params(seed + 1)
    theta[mlp.NH * mlp.NIN:mlp.NH * mlp.NIN + mlp.NH] = rng.normal(scale=0.1, size=mlp.NH)  # b1 != 0
    theta[-1] = 0.3
    return theta, X, y


def test_gradient_matches_central_differences():
    theta, X, y = _batch()
    g, L = mlp.grad(theta, X, y)
    assert abs(L - mlp.loss(theta, X, y)) < 1e-15
    rng = np.random.default_rng(0)
    idx = np.concatenate([rng.choice(mlp.NPARAM, 60, replace=False), [mlp.NPARAM - 1]])
    for i in idx:
        h = 1e-6 * max(1.0, abs(theta[i]))
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss(tp, X, y) - mlp.loss(tm, X, y)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * (abs(g[i]) + 1e-3), (i, fd, g[i])


def test_gelu_tanh_form_close_to_exact_gelu():
    z = np.linspace(-6, 6, 2401)
    exact = 0.5 * z * (1.0 + np.array([math.erf(v / math.sqrt(2.0)) for v in z]))
    # the tanh form approximates z Phi(z) to a few 1e-4 (Hendrycks & Gimpel 2016)
    assert np.max(np.abs(mlp.gelu(z) - exact)) < 1e-3
    assert mlp.gelu(0.0) == 0.0
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.max(np.abs(fd - mlp.gelu_prime(z))) < 1e-8


def test_adam_first_step_is_lr_times_sign():
    theta = np.array([1.0, -2.0, 0.5, 3.0])
    g = np.array([0.3, -4.0, 1e-3, 0.0])
    m = np.zeros(4)
    v = np.zeros(4)
    t1, m1, v1 = mlp.adam(theta, g, m, v, 1, lr=0.01)
    # bias-corrected m/sqrt(v) = g/|g| on the first step (eps aside)
    assert np.allclose((theta - t1)[:3], 0.01 * np.sign(g[:3]), rtol=1e-4)
    assert t1[3] == theta[3]


def test_adam_converges_on_a_quadratic():
    c = np.array([0.7, -1.3])
    th, m, v = np.zeros(2), np.zeros(2), np.zeros(2)
    for t in range(1, 3001):
        th, m, v = mlp.adam(th, th - c, m, v, t, lr=0.01)
    assert np.allclose(th, c, atol=1e-3)


def test_features_are_scale_invariant():
    rng = np.random.default_rng(5)
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    f = w[:, None] * (1 + 0.1 * rng.uniform(-1, 1, size=(19, 9)))
    d = 0.01 * rng.normal(size=(19, 9)) * w[:, None]
    X1, S1 = mlp.features(f, d)
    X2, S2 = mlp.features(f, 4.0 * d)
    assert np.allclose(X1[:, :19], X2[:, :19], rtol=1e-14, atol=0)
    assert np.allclose(X2[:, 19] - X1[:, 19], 2.0 / 8.0)
    assert np.allclose(S2, 4 * S1)
    assert np.allclose(np.max(np.abs(X1[:, :19]), axis=1), 1.0)


def test_zero_weights_give_the_output_bias():
    theta = np.zeros(mlp.NPARAM)
    theta[-1] = -0.25
    o, _ = mlp.forward(theta, np.random.default_rng(1).normal(size=(5, mlp.NIN)))
    assert np.all(o == -0.25)


def test_training_reduces_the_loss():
    rng = np.random.default_rng(11)
    X = rng.uniform(-1, 1, size=(256, mlp.NIN))
    y = 0.5 * X[:, 0] - 0.3 * X[:, 1] * X[:, 2]
    th = mlp.init_params(2)
    m, v = np.zeros_like(th), np.zeros_like(th)
    L0 = mlp.loss(th, X, y)
    for t in range(1, 301):
        g, _ = mlp.grad(th, X, y)
        th, m, v = mlp.adam(th, g, m, v, t, lr=3e-3)
    assert mlp.loss(th, X, y) < 0.1 * L0


def test_hand_set_network_computes_a_known_function():
    """Single paths through the layers: W1[3, 7] picks feature 7 into hidden
    unit 3, W2[5, 3] = 2 feeds unit 5 of layer 2, W3[5] = 1.5, b3 = 0.1; so
    o = 1.5 gelu(2 gelu(X7)) + 0.1 (checked with the exact erf gelu, within
    the tanh form's approximation error)."""
    P = {name: np.zeros(shape) for name, shape in mlp.SHAPES}
    P["W1"][3, 7] = 1.0
    P["W2"][5, 3] = 2.0
    P["W3"][5] = 1.5
    P["b3"][0] = 0.1
    theta = mlp.pack(P)
    X = np.zeros((9, mlp.NIN))
    X[:, 7] = np.linspace(-2, 2, 9)
    X[:, 2] = 5.0  # other features must not leak in
    o, _ = mlp.forward(theta, X)
    ge = lambda z: 0.5 * z * (1.0 + math.erf(z / math.sqrt(2.0)))
    want = np.array([1.5 * ge(2 * ge(v)) + 0.1 for v in X[:, 7]])
    assert np.max(np.abs(o - want)) < 1e-2


def test_series_start_error_is_third_order():
    """alpha_c misses the root of Eq. (entropic) by O(S^3): the truncated
    terms of h start at a^4 M5; checked against the oracle's Newton root."""
    import oracle
    from paper_1612_05404_gb300 import workloads as W
    w = W.D3Q19_WEIGHTS
    for amp in (0.004, 0.01, 0.03):
        f = W.random_populations(40, amp, seed=int(amp * 1e4))
        # Delta of a site: equilibrium at the site's own rho, u minus f
        c, _, _ = oracle.lattice(3)
        out = []
        for i in range(f.shape[1]):
            rho = f[:, i].sum()
            u = (c.T @ f[:, i]) / rho
            d = oracle.feq(3, rho, u) - f[:, i]
            ar, st = oracle.alpha(3, f[:, i], d, 1e-12)
            if st != 0:
                continue
            h0 = oracle.h_prime0(3, f[:, i], d)
            ac = mlp.series_start(f[:, i:i + 1], d[:, None], np.array([h0]))[0]
            S = np.max(np.abs(d / f[:, i]))
            out.append(abs(ac - ar) / S ** 3)
        assert len(out) > 20
        assert max(out) < 2.0, (amp, max(out))
