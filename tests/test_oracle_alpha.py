"""Pins of the oracle's entropic stabiliser: Eq. (entropic) with Eq. (H),
checked in 50-digit decimal arithmetic and by plain bisection."""
import numpy as np
import pytest

import oracle
from tests._hp import H_dec, h_dec


def _state(dim, rng, amp, umax=0.1):
    c, w, _ = oracle.lattice(dim)
    Q = len(w)
    rho = rng.uniform(0.15, 2.2)
    u = np.zeros(3)
    u[:dim] = rng.uniform(-umax, umax, dim)
    f = oracle.feq(dim, rho, u) * np.exp(amp * rng.standard_normal(Q))
    r = f.sum()
    j = f @ c.astype(float)
    d = oracle.feq(dim, r, j / r) - f
    return f, d, w


@pytest.mark.parametrize("dim", [2, 3])
def test_H_closed_forms(dim):
    """Eq. (H), H(f) = sum_p f_p ln(f_p / w_p): zero at the weights, rho ln rho
    at the rest equilibrium f = rho w, and H(f + a D) - H(f) equal to the
    h of Eq. (entropic) (pinned on its own in 50-digit arithmetic)."""
    _, w, _ = oracle.lattice(dim)
    assert abs(oracle.H(dim, w)) < 1e-16
    for rho in (0.16, 1.0, 2.0):
        assert oracle.H(dim, rho * w) == pytest.approx(rho * np.log(rho), rel=1e-14, abs=1e-16)
    rng = np.random.default_rng(60 + dim)
    f, d, _ = _state(dim, rng, 0.05)
    for a in (0.5, 1.7):
        dH = oracle.H(dim, f + a * d) - oracle.H(dim, f)
        assert dH == pytest.approx(oracle.h(dim, f, d, a), rel=1e-9, abs=1e-15)


@pytest.mark.parametrize("dim", [2, 3])
def test_h_log1p_form_equals_H_difference(dim):
    """The oracle's rearranged h(alpha) is H(f + alpha D) - H(f) exactly."""
    rng = np.random.default_rng(10 + dim)
    for amp in (1e-3, 1e-2, 0.1, 0.4):
        f, d, w = _state(dim, rng, amp)
        scale = float(sum(abs(float(x)) for x in f))
        for a in (0.3, 1.0, 1.9, 2.0, 2.4):
            if np.any(f + a * d <= 0):
                continue  # beyond the positivity bound H is undefined
            ref = float(h_dec(f, d, w, a))
            assert abs(oracle.h(dim, f, d, a) - ref) <= 1e-14 * scale


@pytest.mark.parametrize("dim", [2, 3])
def test_alpha_is_the_nontrivial_root(dim):
    """alpha* solves H(f + alpha D) = H(f): sign change of the 50-digit H
    difference across alpha*(1 -+ 1e-9), agreement with bisection to the last
    bits, and alpha* inside the positivity bound."""
    rng = np.random.default_rng(20 + dim)
    n_root = 0
    for amp in (1e-3, 3e-3, 1e-2, 3e-2, 0.1, 0.3):
        for _ in range(6):
            f, d, w = _state(dim, rng, amp)
            a, st = oracle.alpha(dim, f, d)
            if st != 0:
                continue
            n_root += 1
            ab = oracle.alpha_bisect(dim, f, d)
            assert a == pytest.approx(ab, rel=4e-14)
            lo = h_dec(f, d, w, a * (1 - 1e-9))
            hi = h_dec(f, d, w, a * (1 + 1e-9))
            assert lo < 0 < hi
            neg = d < 0
            if neg.any():
                assert a < np.min(-f[neg] / d[neg])
    assert n_root >= 25


def test_alpha_equilibrium_is_bgk():
    """At f = f^eq, alpha = 2 (the BGK value)."""
    for dim in (2, 3):
        f = oracle.feq(dim, 1.3, [0.05, -0.02, 0.01])
        d = oracle.feq(dim, f.sum(), (f @ oracle.lattice(dim)[0].astype(float)) / f.sum()) - f
        a, st = oracle.alpha(dim, f, d)
        assert a == 2.0


def test_alpha_near_equilibrium_tends_to_two():
    """For a small deviation at rest the root approaches 2 (the quadratic
    term of h dominates): |alpha - 2| shrinks with the deviation."""
    rng = np.random.default_rng(30)
    prev = None
    for amp in (1e-1, 1e-2, 1e-3):
        errs = []
        for _ in range(5):
            f, d, w = _state(3, rng, amp, umax=0.0)
            a, st = oracle.alpha(3, f, d)
            assert st == 0
            errs.append(abs(a - 2.0))
        m = max(errs)
        if prev is not None:
            assert m < 0.5 * prev
        prev = m


@pytest.mark.parametrize("dim", [2, 3])
def test_h_theorem(dim):
    """Post-collision H never exceeds pre-collision H for beta in (0, 1]:
    H(f + alpha beta D) <= H(f) (convexity of h between its two zeros)."""
    rng = np.random.default_rng(40 + dim)
    for amp in (1e-2, 0.1, 0.3):
        for _ in range(4):
            f, d, w = _state(dim, rng, amp)
            a, st = oracle.alpha(dim, f, d)
            if st != 0:
                continue
            for beta in (0.2, 0.5, 0.9, 1.0):
                dh = h_dec(f, d, w, a * beta)
                assert float(dh) <= 1e-14 * f.sum()


def test_no_root_falls_back_to_bgk():
    """When h'(0) >= 0 (possible with the polynomial equilibrium at finite
    velocity and tiny non-equilibrium) no positive alpha keeps H from rising;
    the oracle falls back to alpha = 2 and reports it."""
    rng = np.random.default_rng(50)
    c, w, _ = oracle.lattice(3)
    found = 0
    for _ in range(4000):
        u = rng.uniform(-0.15, 0.15, 3)
        f = oracle.feq(3, 1.0, u) * np.exp(3e-6 * rng.standard_normal(19))
        r = f.sum()
        d = oracle.feq(3, r, (f @ c.astype(float)) / r) - f
        a, st = oracle.alpha(3, f, d)
        if st == 2:
            found += 1
            assert a == 2.0
            # the 50-digit derivative at 0 is non-negative: h(eps) > 0
            assert h_dec(f, d, w, 1e-6) > 0
            if found >= 3:
                break
    assert found >= 1
