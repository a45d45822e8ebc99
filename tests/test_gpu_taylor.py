"""The leaky-dielectric drop in a uniform field (the 64^3 drop-in-field
workload, E0 swept over 1e-4 .. 1e-3, 5000 steps on the GPU): the trend of
its small deformation against Taylor's theory (G. I. Taylor 1966, "Studies in
electrohydrodynamics I", Proc. R. Soc. A 291; the discriminating function in
the form of Melcher & Taylor 1969).

For a drop of radius a, conductivity, permittivity and viscosity ratios
(drop over medium) R, S and lambda, in a field E0, Taylor's deformation
D = (L - B)/(L + B) (L along the field, B across) is, to first order in the
electric capillary number Ca = eps_medium E0^2 a / gamma,
    D = 9/16 Ca Phi / (2 + R)^2,
    Phi = R^2 + 1 - 2 S + 3 (R - S)(2 + 3 lambda) / (5 (1 + lambda)),
so D grows linearly with E0^2, prolate where Phi > 0 and oblate where
Phi < 0 (Phi = (R - 1)^2 >= 0 for R = S, the perfect-dielectric limit;
Phi -> R^2 for a conducting drop, D -> 9 Ca / 16). Here R = 10, S = 2 and
lambda = rho_L / rho_V = 12.5 (equal kinematic viscosity at rest), so
Phi = 111 > 0: prolate, D - D(0) proportional to E0^2. The magnitude is
not checked: the lattice surface tension, the confinement between the
electrodes and the qE form of the force all enter it."""
import numpy as np
import pytest

from paper_1612_05404_gb300 import workloads as W


def _deformation(rho, n, thr=1.08):
    """D = (L - B)/(L + B) from the second moments of the liquid (rho above
    thr, weighted by rho - thr): L^2 ~ <(z - z_c)^2> along the field (z), B^2
    ~ the mean of <(x - x_c)^2> and <(y - y_c)^2>."""
    r = rho.reshape(n, n, n)  # (z, y, x)
    w = np.clip(r - thr, 0.0, None)
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    m = w.sum()
    c = [(w * a).sum() / m for a in (z, y, x)]
    izz, iyy, ixx = [(w * (a - ca) ** 2).sum() / m for a, ca in zip((z, y, x), c)]
    L, B = np.sqrt(izz), np.sqrt(0.5 * (ixx + iyy))
    return (L - B) / (L + B)


def _taylor_phi(R, S, lam):
    return R * R + 1.0 - 2.0 * S + 3.0 * (R - S) * (2.0 + 3.0 * lam) / (5.0 * (1.0 + lam))


def test_taylor_phi_limits():
    """The discriminating function's textbook limits (no GPU work): the
    perfect dielectric (R = S) and the conducting drop (R -> infinity)."""
    for S in (0.5, 2.0, 5.0):
        assert abs(_taylor_phi(S, S, 3.0) - (S - 1.0) ** 2) < 1e-12
    R = 1e6
    assert abs(9.0 / 16.0 * _taylor_phi(R, 2.0, 1.0) / (2.0 + R) ** 2 - 9.0 / 16.0) < 1e-5


@pytest.mark.gpu
def test_drop_deformation_follows_taylor_trend():
    from paper_1612_05404_gb300 import elbm
    E0s = list(W.E0_SWEEP) + [0.0]
    sims = []
    for E0 in E0s:
        cfg, fields = W.drop_in_field(E0=E0, precision="fp32")
        cfg.update(alpha_precision="fp32", autotune=1)
        sims.append(elbm.Sim(cfg, fields))
    cfg = W.drop_in_field(E0=1e-3, precision="fp32")[0]
    eps_l = 1.0 + cfg["eps_kappa"] * W.RHO_L / cfg["rho0"]
    eps_v = 1.0 + cfg["eps_kappa"] * W.RHO_V / cfg["rho0"]
    phi_t = _taylor_phi(cfg["sigma_liq"] / cfg["sigma_gas"], eps_l / eps_v, W.RHO_L / W.RHO_V)
    assert phi_t > 0.0  # Taylor: prolate
    batch = elbm.Batch(sims, pipeline=True, span=10)
    assert batch.step(5000) == elbm.OK
    batch.close()
    n = cfg["shape"][0]
    D = np.array([_deformation(s.get("rho"), n) for s in sims])
    for s in sims:
        d = s.diag()
        assert d["max_h_error"] <= 1e-10 and d["n_guard_failed"] == 0
        s.close()
    e2 = np.array(E0s[:4]) ** 2
    slope, icpt = np.polyfit(e2, D[:4], 1)
    resid = D[:4] - (icpt + slope * e2)
    span = D[3] - D[0]
    print("Taylor: Phi = %.1f, D = %s, D(E0=0) = %.3e, fit D = %.4e + %.4e E0^2, residuals %s"
          % (phi_t, D[:4], D[4], icpt, slope, resid))
    # prolate and growing with the field, as Phi > 0 says
    assert slope > 0.0 and np.all(np.diff(D[:4]) > 0.0)
    # linear in E0^2: residuals of the straight line within 2 % of the
    # deformation the sweep adds, and the line meets the field-free drop
    assert np.max(np.abs(resid)) <= 0.02 * span, resid
    assert abs(icpt - D[4]) <= 0.02 * span, (icpt, D[4])
