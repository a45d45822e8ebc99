"""Pins of the oracle's non-Newtonian part: matrix 2-norm (Sec. II B),
Carreau law Eq. (carreau) inside the root of Eq. (strain2), and a Poiseuille
channel whose shear stress is fixed by force balance."""
import numpy as np
import pytest
from scipy.optimize import brentq

import oracle
from paper_1612_05404_gb300 import workloads as W


def test_spectral_norm_matches_eigvalsh():
    rng = np.random.default_rng(60)
    for dim in (2, 3):
        for _ in range(200):
            A = rng.standard_normal((dim, dim)) * 10.0 ** rng.uniform(-6, 1)
            S = 0.5 * (A + A.T)
            ref = np.max(np.abs(np.linalg.eigvalsh(S)))
            assert oracle.spectral_norm(dim, S) == pytest.approx(ref, rel=1e-13)
    # diagonal and rank-one special cases
    assert oracle.spectral_norm(3, np.diag([1.0, -3.0, 2.0])) == 3.0
    v = np.array([1.0, 2.0, -2.0])
    assert oracle.spectral_norm(3, np.outer(v, v)) == pytest.approx(9.0, rel=1e-14)


def _carreau_cfg(**kw):
    cfg = W.base_params(nu0=1.0 / 6, nu_inf=1.0 / 60, n_carreau=0.5)
    cfg["lambda"] = 20.0
    cfg.update(kw)
    return cfg


def test_carreau_newtonian_limits():
    cfg = _carreau_cfg(n_carreau=1.0)
    for Pn in (0.0, 1e-4, 0.3):
        g, nu = oracle.carreau(cfg, Pn, 2.0, 1.0)
        assert nu == cfg["nu0"]
    g, nu = oracle.carreau(_carreau_cfg(), 0.0, 2.0, 1.5)
    assert g == 0.0 and nu == 1.0 / 6


def test_carreau_root_solves_strain_equation():
    """gdot = Pi alpha beta(nu(gdot)) / (rho c_s^2), nu by the Carreau law,
    beta = c_s^2/(2 nu + c_s^2); the residual is at rounding level and nu
    lies between nu_inf and nu0."""
    cfg = _carreau_cfg()
    rng = np.random.default_rng(61)
    for _ in range(200):
        Pn = 10 ** rng.uniform(-7, -0.5)
        a = rng.uniform(1.5, 2.5)
        rho = rng.uniform(0.15, 2.2)
        g, nu = oracle.carreau(cfg, Pn, a, rho)
        nu_ref = cfg["nu_inf"] + (cfg["nu0"] - cfg["nu_inf"]) * (1 + (cfg["lambda"] * g) ** 2) ** (
            (cfg["n_carreau"] - 1) / 2)
        beta = (1 / 3) / (2 * nu_ref + 1 / 3)
        assert nu == pytest.approx(nu_ref, rel=1e-13)
        assert g == pytest.approx(Pn * a * beta / (rho / 3), rel=1e-12)
        assert cfg["nu_inf"] <= nu <= cfg["nu0"]


def _channel(n_carreau, lam, alpha_mode, steps=3000):
    """2-D channel, walls at y = -1/2 and ny - 1/2, driven by a uniform force
    F = q E_ext with a uniform xi-form bulk charge on a uniform fluid."""
    nx, ny = 2, 20
    cfg = W.base_params(dim=2, shape=(nx, ny, 1), G=0.0, Gw=0.0, charge_model="xi",
                        xi_b=1e-2, xi_s=0.0, E_ext=(3.35e-3, 0.0, 0.0), phi_axis=0,
                        face_bc=["periodic", "periodic", "wall", "wall", "periodic", "periodic"],
                        phi_bc=["periodic", "periodic", "neumann", "neumann", "periodic", "periodic"],
                        nu0=1.0 / 6, nu_inf=1.0 / 60, n_carreau=n_carreau,
                        alpha_mode=alpha_mode)
    cfg["lambda"] = lam
    sim = oracle.Sim(cfg, dict(mask=np.zeros(nx * ny, np.uint8), rho=np.full(nx * ny, 2.0)))
    sim.step(steps)
    theta = 0.5 * (1 + np.tanh((2.0 - 1.0) / 0.1))
    F = 1e-2 * 2.0 * theta * 3.35e-3
    return sim, F, ny


def test_poiseuille_newtonian_profile():
    """Steady Newtonian channel: u(y) = F y'(H - y')/(2 rho nu), y' = y + 1/2."""
    sim, F, ny = _channel(1.0, 0.0, "bgk")
    u = sim.u.reshape(ny, 2, 3)[:, 0, 0]
    yp = np.arange(ny) + 0.5
    ref = F * yp * (ny - yp) / (2 * 2.0 * (1 / 6))
    assert np.allclose(u, ref, rtol=2e-3, atol=2e-3 * ref.max())


def test_poiseuille_carreau_viscosity_from_force_balance():
    """Shear-thinning channel: the local shear stress is fixed by force
    balance, rho nu(gdot) gdot = F |H/2 - y'|, whatever the rheology; the
    oracle's nu (through Pi, the 2-norm, Eq. strain2 and Eq. carreau) must
    match the nu that solves it."""
    lam, n = 1500.0, 0.5
    sim, F, ny = _channel(n, lam, "entropic", steps=4000)
    nu_o = sim.nu.reshape(ny, 2)[:, 0]
    yp = np.arange(ny) + 0.5
    nu0, nui = 1 / 6, 1 / 60

    def nu_c(g):
        return nui + (nu0 - nui) * (1 + (lam * g) ** 2) ** ((n - 1) / 2)

    checked = 0
    for k in range(ny):
        tau = F * abs(ny / 2 - yp[k])
        if tau < 0.3 * F * ny / 2:
            continue  # near the centre line the shear vanishes
        g = brentq(lambda g: 2.0 * nu_c(g) * g - tau, 0.0, 1.0, xtol=1e-16)
        assert nu_o[k] == pytest.approx(nu_c(g), rel=0.03)
        checked += 1
    assert checked >= 10
    assert nu_o.min() < 0.75 * nu0  # genuinely in the shear-thinning range
