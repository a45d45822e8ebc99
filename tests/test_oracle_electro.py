"""Pins of the oracle's electrostatics: the Poisson solve (Sec. II) against a
direct solve and a manufactured solution, Gauss's law and the paper's |E| on
the 2-D charged drop, the charge models Eqs. (surface-q2)/(surface-q3) with
the curvature K, and the transported charge relaxing with time constant
eps/sigma."""
import numpy as np
import pytest

import oracle
from paper_1612_05404_gb300 import workloads as W


def _dense_vs_sor(cfg, mask, rho, qn):
    A, b, index = oracle.poisson_system(cfg, mask, rho, qn)
    x = np.linalg.solve(A, b)
    ref = np.zeros(mask.size)
    ref[index >= 0] = x[index[index >= 0]]
    phi, it, res = oracle.poisson_solve(cfg, mask, rho, qn)
    return phi, ref, it, res


def test_poisson_periodic_matches_direct_solve():
    shape = (6, 4, 6)
    N = 144
    cfg = W.base_params(shape=shape, charge_model="xi", poisson_tol=1e-14, eps_kappa=0.7)
    rng = np.random.default_rng(80)
    rho = rng.uniform(0.16, 2.0, N)
    q = rng.standard_normal(N)
    qn = q - q.mean()
    phi, ref, it, res = _dense_vs_sor(cfg, np.zeros(N, np.uint8), rho, qn)
    assert res <= 1e-14 and it > 0
    assert np.allclose(phi, ref - ref.mean(), rtol=0, atol=1e-11 * np.abs(ref).max())


def test_poisson_odd_periodic_extents_match_direct_solve():
    """Odd periodic extents (5 x 7 x 3, every axis periodic): red-black cannot
    colour them (the two sites across the wrap share a parity), the sweep takes
    the three-colour ordering; its converged potential is the direct solution
    of the same discrete system."""
    shape = (5, 7, 3)
    N = 105
    cfg = W.base_params(shape=shape, charge_model="xi", poisson_tol=1e-14, eps_kappa=0.7)
    rng = np.random.default_rng(82)
    rho = rng.uniform(0.16, 2.0, N)
    q = rng.standard_normal(N)
    qn = q - q.mean()
    phi, ref, it, res = _dense_vs_sor(cfg, np.zeros(N, np.uint8), rho, qn)
    assert res <= 1e-14 and it > 0
    assert np.allclose(phi, ref - ref.mean(), rtol=0, atol=1e-11 * np.abs(ref).max())


def test_poisson_odd_periodic_with_electrodes_matches_direct_solve():
    """An odd periodic extent beside even ones and Dirichlet electrodes (7 x 4
    x 5, periodic in x and y, electrodes on the z faces, one conductor node)."""
    shape = (7, 4, 5)
    N = 140
    cfg = W.base_params(shape=shape, charge_model="xi", poisson_tol=1e-14,
                        face_bc=["periodic"] * 4 + ["wall", "wall"],
                        phi_bc=["periodic"] * 4 + ["dirichlet", "dirichlet"],
                        phi_lo=0.1, phi_hi=-0.4, phi_solid=0.05)
    rng = np.random.default_rng(83)
    mask = np.zeros(N, np.uint8)
    mask[61] = oracle.SOLID
    rho = rng.uniform(0.16, 2.0, N)
    qn = rng.standard_normal(N) * (mask == 0)
    phi, ref, it, res = _dense_vs_sor(cfg, mask, rho, qn)
    fl = mask == 0
    assert np.allclose(phi[fl], ref[fl], rtol=0, atol=1e-11 * np.abs(ref).max())


def test_three_colour_sweep_is_independent_of_the_thread_count():
    """A site updates from sites of other colours only, so the result of a
    sweep does not depend on how the sites of a colour are split over
    threads: two fixed sweeps on 1 and 4 threads agree bit for bit (with two
    colours on an odd periodic extent, the two sites across the wrap would
    read each other while being written)."""
    shape = (9, 5, 7)
    N = 315
    cfg = W.base_params(shape=shape, charge_model="xi", poisson_fixed_sweeps=2, eps_kappa=0.7)
    rng = np.random.default_rng(84)
    rho = rng.uniform(0.16, 2.0, N)
    q = rng.standard_normal(N)
    qn = q - q.mean()
    mask = np.zeros(N, np.uint8)
    n0 = oracle.set_threads(0)
    try:
        out = []
        for t in (1, 4):
            oracle.set_threads(t)
            out.append(oracle.poisson_solve(cfg, mask, rho, qn)[0])
    finally:
        oracle.set_threads(n0)
    assert np.array_equal(out[0], out[1])


def test_poisson_point_charge_matches_fourier_green_function():
    """Uniform permittivity on a periodic 12 x 10 x 8 lattice (eps = 1 +
    kappa rho with rho uniform): the 7-point operator is diagonal in Fourier
    space, eigenvalue
    -eps lambda(k), lambda(k) = sum_a 2 (1 - cos(2 pi k_a / n_a)). A point
    charge with its neutralising background then has the potential
    phi_hat(k) = q_hat(k) / (eps lambda(k)) (k != 0, zero mean), computed
    here by numpy's FFT: the oracle's SOR potential matches it."""
    nx, ny, nz = 12, 10, 8
    N = nx * ny * nz
    kap = 0.7
    cfg = W.base_params(shape=(nx, ny, nz), charge_model="xi", poisson_tol=1e-14, eps_kappa=kap)
    rho = np.full(N, 1.3)
    eps = 1.0 + kap * 1.3
    q = np.zeros(N)
    q[3 + nx * (4 + ny * 2)] = 1.0
    qn = q - q.mean()
    phi, it, res = oracle.poisson_solve(cfg, np.zeros(N, np.uint8), rho, qn)
    assert res <= 1e-14 and it > 0
    kz, ky, kx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    lam = (2 * (1 - np.cos(2 * np.pi * kx / nx)) + 2 * (1 - np.cos(2 * np.pi * ky / ny))
           + 2 * (1 - np.cos(2 * np.pi * kz / nz)))
    qh = np.fft.fftn(qn.reshape(nz, ny, nx))
    ph = np.zeros_like(qh)
    nzk = lam > 0
    ph[nzk] = qh[nzk] / (eps * lam[nzk])  # div(eps grad phi) = -q  =>  eps lambda phi_hat = q_hat
    ref = np.real(np.fft.ifftn(ph)).reshape(-1)
    assert np.allclose(phi, ref - ref.mean(), rtol=0, atol=1e-11 * np.abs(ref).max())


def test_poisson_2d_point_charge_matches_fourier_green_function():
    """The same pin for the paper's 2-D lattice (nz = 1, dim 2; the odd
    periodic extent 13 puts the sweep on three colours): the 5-point
    operator, eigenvalue -eps lambda(k) with lambda(k) = 2 (1 - cos(2 pi
    k_x / n_x)) + 2 (1 - cos(2 pi k_y / n_y)), two charges of unequal sign
    and size with their neutralising background."""
    nx, ny = 13, 10
    N = nx * ny
    kap = 1.0
    cfg = W.base_params(dim=2, shape=(nx, ny, 1), phi_axis=0, charge_model="xi", poisson_tol=1e-14,
                        eps_kappa=kap)
    rho = np.full(N, 0.4)
    eps = 1.0 + kap * 0.4
    q = np.zeros(N)
    q[5 + nx * 3] = 1.0
    q[9 + nx * 7] = -0.4
    qn = q - q.mean()
    phi, it, res = oracle.poisson_solve(cfg, np.zeros(N, np.uint8), rho, qn)
    assert res <= 1e-14 and it > 0
    ky, kx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    lam = 2 * (1 - np.cos(2 * np.pi * kx / nx)) + 2 * (1 - np.cos(2 * np.pi * ky / ny))
    qh = np.fft.fft2(qn.reshape(ny, nx))
    ph = np.zeros_like(qh)
    nzk = lam > 0
    ph[nzk] = qh[nzk] / (eps * lam[nzk])
    ref = np.real(np.fft.ifft2(ph)).reshape(-1)
    assert np.allclose(phi, ref - ref.mean(), rtol=0, atol=1e-11 * np.abs(ref).max())


def test_step_potential_solves_the_neutralised_problem():
    """Inside a time step (Sec. II C) the potential solves div(eps grad phi) =
    -(q - <q>): the free charge of the step less its mean (the uniform
    background of reading 17). With uniform eps on a periodic lattice that
    solution is the Fourier one, phi_hat = q_hat / (eps lambda(k)), k != 0,
    taken here from the step's own charge."""
    nx, ny = 20, 16
    cfg = W.base_params(dim=2, shape=(nx, ny, 1), phi_axis=0, charge_model="conserved", Q_b=0.3, Q_s=0.9,
                        eps_kappa=0.0, poisson_tol=1e-13, poisson_check_every=1)
    rho = W.drop_profile((nx, ny, 1), 5.0, dim=2)
    sim = oracle.Sim(cfg, dict(mask=np.zeros(nx * ny, np.uint8), rho=rho))
    sim.step(1)
    q = sim.q
    assert abs(q.sum() - 1.2) < 1e-12 and q.min() >= 0.0
    ky, kx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    lam = 2 * (1 - np.cos(2 * np.pi * kx / nx)) + 2 * (1 - np.cos(2 * np.pi * ky / ny))
    qh = np.fft.fft2((q - q.mean()).reshape(ny, nx))
    ph = np.zeros_like(qh)
    ph[lam > 0] = qh[lam > 0] / lam[lam > 0]
    ref = np.real(np.fft.ifft2(ph)).reshape(-1)
    assert np.allclose(sim.phi, ref - ref.mean(), rtol=0, atol=1e-10 * np.abs(ref).max())


def test_poisson_dirichlet_and_conductors_match_direct_solve():
    shape = (6, 4, 5)
    N = 120
    cfg = W.base_params(shape=shape, charge_model="xi", poisson_tol=1e-14,
                        face_bc=["periodic", "periodic", "wall", "wall", "wall", "wall"],
                        phi_bc=["periodic", "periodic", "neumann", "neumann", "dirichlet", "dirichlet"],
                        phi_lo=0.2, phi_hi=-0.5, phi_solid=0.1)
    rng = np.random.default_rng(81)
    mask = np.zeros(N, np.uint8)
    mask[[13, 50, 77]] = oracle.SOLID
    rho = rng.uniform(0.16, 2.0, N)
    qn = rng.standard_normal(N) * (mask == 0)
    phi, ref, it, res = _dense_vs_sor(cfg, mask, rho, qn)
    fl = mask == 0
    assert np.allclose(phi[fl], ref[fl], rtol=0, atol=1e-11 * np.abs(ref).max())


def test_poisson_manufactured_second_order():
    """phi = sin(2pi x/n) sin(2pi y/n) sin(pi (z+1)/(n+1)) + linear(z) with
    eps = 1 + kappa rho(x, y) smooth: the discrete solution converges to it at
    second order (error ratio ~4 per halving of the spacing)."""
    errs = []
    for n in (8, 16):
        shape = (n, n, n)
        x, y, z = [a.reshape(-1) for a in np.meshgrid(np.arange(n), np.arange(n), np.arange(n),
                                                       indexing="xy")]
        x, y, z = (np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")[::-1])
        x, y, z = x.reshape(-1).astype(float), y.reshape(-1).astype(float), z.reshape(-1).astype(float)
        kx = ky = 2 * np.pi / n
        kz = np.pi / (n + 1)
        lo, hi = 0.3, -0.7
        kap = 0.5
        rho = 1.0 + 0.5 * np.cos(kx * x) * np.cos(ky * y)
        eps = 1.0 + kap * rho
        ex = -kap * 0.5 * kx * np.sin(kx * x) * np.cos(ky * y)
        ey = -kap * 0.5 * ky * np.cos(kx * x) * np.sin(ky * y)
        S = np.sin(kx * x) * np.sin(ky * y) * np.sin(kz * (z + 1))
        phi_ex = S + lo + (z + 1) * (hi - lo) / (n + 1)
        px = kx * np.cos(kx * x) * np.sin(ky * y) * np.sin(kz * (z + 1))
        py = ky * np.sin(kx * x) * np.cos(ky * y) * np.sin(kz * (z + 1))
        lap = -(kx ** 2 + ky ** 2 + kz ** 2) * S
        q = -(eps * lap + ex * px + ey * py)
        cfg = W.base_params(shape=shape, charge_model="xi", poisson_tol=1e-13, eps_kappa=kap,
                            face_bc=["periodic"] * 4 + ["wall", "wall"],
                            phi_bc=["periodic"] * 4 + ["dirichlet", "dirichlet"],
                            phi_lo=lo, phi_hi=hi)
        phi, it, res = oracle.poisson_solve(cfg, np.zeros(n ** 3, np.uint8), rho, q)
        errs.append(np.abs(phi - phi_ex).max())
    assert 3.0 < errs[0] / errs[1] < 5.5


def test_conserved_charge_totals(paper):
    """Eq. (surface-q2): sum q = Q_b + Q_s exactly, split in the ratio
    Q_s/Q_b = 10, on the paper's 2-D drop; and each total sits where its
    term puts it: the bulk charge (rho theta(rho)) fills the liquid's
    interior and is absent from the gas, the surface charge (|grad rho|^2)
    lies on the interface (measured: bulk minimum 3x the interface mean,
    gas 1e-8 of it; surface charge inside 1.5 % of its interface peak)."""
    cfg, fl = W.paper_drop_2d(n=96, radius=20.0)
    rho = fl["rho"]
    q, K, sums = oracle.charge_field(cfg, fl["mask"], rho)
    assert q.sum() == pytest.approx(paper["Q_total"]["value"], rel=1e-13)
    qb, _, _ = oracle.charge_field(dict(cfg, Q_s=0.0), fl["mask"], rho)
    assert (q.sum() - qb.sum()) / qb.sum() == pytest.approx(paper["Qs_over_Qb"]["value"], rel=1e-12)
    qs, _, _ = oracle.charge_field(dict(cfg, Q_b=0.0), fl["mask"], rho)
    bulk, inter, gas = rho > 1.95, (rho > 0.6) & (rho < 1.5), rho < 0.2
    assert qb[bulk].min() > 2.0 * qb[inter].mean() and qb[gas].max() < 1e-6 * qb[bulk].min()
    assert qs[bulk].max() < 0.05 * qs[inter].max()


def test_xi_form_is_linear_in_coefficients():
    cfg, fl = W.paper_drop_2d(n=64, radius=15.0)
    c1 = dict(cfg, charge_model="xi", xi_b=1e-4, xi_s=0.0)
    c2 = dict(cfg, charge_model="xi", xi_b=0.0, xi_s=6e-2)
    c3 = dict(cfg, charge_model="xi", xi_b=1e-4, xi_s=6e-2)
    q1 = oracle.charge_field(c1, fl["mask"], fl["rho"])[0]
    q2 = oracle.charge_field(c2, fl["mask"], fl["rho"])[0]
    q3 = oracle.charge_field(c3, fl["mask"], fl["rho"])[0]
    assert np.allclose(q3, q1 + q2, rtol=1e-14, atol=0)
    rho = fl["rho"]
    th = 0.5 * (1 + np.tanh((rho - 1.0) / 0.1))
    assert np.allclose(q1, 1e-4 * rho * th, rtol=1e-13)


def test_surface_charge_curvature_exponent():
    """Eq. (surface-q3)'s surface term xi_s |grad rho|^2 (1 + (K/K_d)^(1/4)),
    pinned without |grad rho|^2 or K: at a site with K > 0, q(K_d) with
    xi_b = 0, xi_s = 1 for K_d = 1, 16, 256 gives
    (q(1) - q(16)) / (q(16) - q(256)) = 16^(1/4) = 2 exactly, whatever the
    gradient and the curvature; any other exponent p gives 16^p."""
    n = 40
    rho = W.drop_profile((n, n, 1), 9.0, dim=2)
    mask = np.zeros(n * n, np.uint8)
    qs = []
    for kd in (1.0, 16.0, 256.0):
        cfg = W.base_params(dim=2, shape=(n, n, 1), phi_axis=0, charge_model="xi", xi_b=0.0, xi_s=1.0,
                            K_d=kd)
        q, K, _ = oracle.charge_field(cfg, mask, rho)
        qs.append(q)
    sel = (K > 1e-3) & (qs[2] > 1e-4)
    assert sel.sum() > 50
    ratio = (qs[0][sel] - qs[1][sel]) / (qs[1][sel] - qs[2][sel])
    assert np.allclose(ratio, 2.0, rtol=1e-9, atol=0)


def test_mean_curvature_circle_and_sphere():
    """K = -div(grad rho/|grad rho|) equals 1/R on a circle and 2/R on a
    sphere at the interface (positive on convex drops)."""
    cfg, fl = W.paper_drop_2d(n=128, radius=30.0)
    _, K, _ = oracle.charge_field(cfg, fl["mask"], fl["rho"])
    n = 128
    x = np.arange(n) - 63.5
    d = np.sqrt(x[None, :] ** 2 + x[:, None] ** 2).reshape(-1)
    sel = np.abs(d - 30.0) < 0.5
    assert K[sel].mean() == pytest.approx(1 / 30.0, rel=0.02)
    n3 = 40
    cfg3 = W.base_params(shape=(n3, n3, n3), charge_model="conserved", Q_s=1.0)
    rho3 = W.drop_profile((n3, n3, n3), 12.0)
    _, K3, _ = oracle.charge_field(cfg3, np.zeros(n3 ** 3, np.uint8), rho3)
    g = np.arange(n3) - (n3 - 1) / 2
    d3 = np.sqrt(g[None, None, :] ** 2 + g[None, :, None] ** 2 + g[:, None, None] ** 2).reshape(-1)
    sel3 = np.abs(d3 - 12.0) < 0.5
    assert K3[sel3].mean() == pytest.approx(2 / 12.0, rel=0.03)


@pytest.mark.slow
def test_paper_drop_field_gauss_law_and_boundary_value(paper):
    """The paper's 2-D charged drop (320^2, R = 40, Q = 2.13, Q_s/Q_b = 10,
    eps = 1 + rho, neutralised): outside the drop |E| follows Gauss's law,
    |E| = Q_enc/(2 pi r eps_V), and the paper's boundary value 3.5e-3 lies
    within the range of |E| across the interface."""
    cfg, fl = W.paper_drop_2d()
    cfg["poisson_tol"] = 1e-8
    n = 320
    q, _, _ = oracle.charge_field(cfg, fl["mask"], fl["rho"])
    qm = q.mean()
    phi, it, res = oracle.poisson_solve(cfg, fl["mask"], fl["rho"], q - qm, qmean=qm)
    E = oracle.efield(cfg, fl["mask"], phi)
    Em = np.sqrt((E ** 2).sum(1))
    x = np.arange(n) - 159.5
    d = np.sqrt(x[None, :] ** 2 + x[:, None] ** 2).reshape(-1)
    Q = paper["Q_total"]["value"]
    eps_v = 1.0 + fl["rho"][0]
    for r in (60.0, 80.0):
        sel = np.abs(d - r) < 0.5
        q_enc = Q * (1.0 - np.pi * r ** 2 / n ** 2)
        assert Em[sel].mean() == pytest.approx(q_enc / (2 * np.pi * r * eps_v), rel=0.02)
    band = (d > 37.0) & (d < 45.0)
    Eb = paper["E_boundary"]["value"]
    assert Em[band].min() < Eb < Em[band].max()


def _decay_run(n=16, steps=30, sigma=0.06, kappa=1.0, Dq=1e-3, amp=1e-6):
    shape = (n, 4, 4)
    N = n * 16
    cfg = W.base_params(shape=shape, G=0.0, Gw=0.0, charge_model="transport",
                        sigma_liq=sigma, sigma_gas=sigma, eps_kappa=kappa, Dq=Dq,
                        poisson_tol=1e-13)
    x = np.tile(np.arange(n), 16).astype(float)
    q0 = amp * np.sin(2 * np.pi * x / n)
    sim = oracle.Sim(cfg, dict(mask=np.zeros(N, np.uint8), rho=np.full(N, 2.0), q=q0))
    qs = []
    for _ in range(steps):
        qs.append(sim.g.reshape(7, N).sum(0)[:n].copy())
        sim.step()
    return np.array(qs), cfg


def test_transport_mode_matches_linear_mode_dynamics():
    """Uniform medium at rest: a single Fourier mode of the transported charge
    evolves by the 7x7 linear map of the D3Q7 collision with the Ohmic source
    R = sigma Lphi = -(sigma/eps) q (Poisson eps Lphi = -q) followed by
    streaming. Computed here in Fourier space, independently of the oracle's
    site loops."""
    n, steps, sigma, kappa, Dq = 16, 30, 0.06, 1.0, 1e-3
    qs, cfg = _decay_run(n, steps, sigma, kappa, Dq)
    eps = 1.0 + kappa * 2.0
    tau = 0.5 + Dq / 0.25
    w = np.array([0.25] + [0.125] * 6)
    cx = np.array([0, 1, -1, 0, 0, 0, 0])
    k = 2 * np.pi / n
    one = np.ones(7)
    C = np.eye(7) - (np.eye(7) - np.outer(w, one)) / tau - (sigma / eps) * np.outer(w, one)
    M = np.diag(np.exp(-1j * k * cx)) @ C
    a = w * (-1j) * 1e-6
    xs = np.arange(n)
    for t in range(steps):
        qt = np.real(one @ a * np.exp(1j * k * xs))
        assert np.allclose(qs[t], qt, rtol=0, atol=1e-9 * 1e-6)
        a = M @ a


def test_transport_relaxation_time_constant():
    """Charge relaxation in a uniform conductor: the amplitude decays as
    exp(-t/tau_e) with tau_e = eps/sigma (plus the small diffusive rate
    D k^2)."""
    n, steps = 16, 30
    for sigma, kappa in ((0.06, 1.0), (0.02, 0.5)):
        qs, _ = _decay_run(n, steps, sigma, kappa, 1e-3)
        amp = np.abs(qs).max(1)
        rate = -np.polyfit(np.arange(steps), np.log(amp), 1)[0]
        eps = 1.0 + 2.0 * kappa
        expect = sigma / eps + 0.25 * (4e-3) * (2 * np.pi / n) ** 2
        assert rate == pytest.approx(-np.log(1 - expect), rel=0.02)


def test_transport_advects_charge_with_the_flow():
    """A Gaussian of transported charge in a uniform flow u (no conduction,
    no Shan-Chen coupling): the equilibrium w q (1 + c.u/c_s,q^2) carries the
    flux q u, and the global flux is conserved by streaming and kept by the
    relaxation, so the charge's first moment advances by exactly Q u per step
    (the centroid moves at u; diffusion only widens it). A wrong sign or
    factor in the c.u/c_s,q^2 term fails. The charge is small (1e-6), so its
    electric force leaves the flow uniform to O(1e-12). The Gaussian starts
    at the middle of a 64-site periodic axis so that nothing of it (nor of
    the scheme's ripples near tau_q = 1/2) crosses the wrap, where a
    population would move the first moment by the axis length."""
    n, steps, ux = 64, 60, 0.05
    shape = (n, 4, 4)
    N = n * 16
    # (one SOR sweep per step: with no conduction the potential enters only
    # through the force q E, negligible at this charge)
    cfg = W.base_params(shape=shape, G=0.0, Gw=0.0, charge_model="transport", sigma_liq=0.0,
                        sigma_gas=0.0, Dq=1e-2, poisson_fixed_sweeps=1)
    x = np.tile(np.arange(n), 16).astype(float)
    q0 = 1e-6 * np.exp(-0.5 * ((x - 32.0) / 2.0) ** 2)
    u0 = np.zeros((N, 3))
    u0[:, 0] = ux
    sim = oracle.Sim(cfg, dict(mask=np.zeros(N, np.uint8), rho=np.full(N, 2.0), q=q0, u=u0.reshape(-1)))

    def moments():
        q = sim.g.reshape(7, N).sum(0)
        return q.sum(), (q * x).sum()

    Q0, M0 = moments()
    sim.step(steps)
    Q1, M1 = moments()
    assert abs(Q1 - Q0) <= 1e-14 * Q0
    assert abs(M1 - M0 - steps * ux * Q0) <= 1e-6 * steps * ux * Q0, (M1 - M0, steps * ux * Q0)


def test_uniform_field_on_neutral_fluid_exerts_no_force():
    shape = (4, 4, 4)
    cfg = W.base_params(shape=shape, G=0.0, Gw=0.0, charge_model="xi", xi_b=0.0, xi_s=0.0,
                        E_ext=(0.3, -0.1, 0.2))
    sim = oracle.Sim(cfg, dict(mask=np.zeros(64, np.uint8), rho=np.full(64, 1.5)))
    r0, j0 = sim.moments()
    sim.step()
    r1, j1 = sim.moments()
    assert np.abs(j1).max() < 1e-16


def _force_from_step(sim):
    """Body force per site from one oracle step started at rest: the
    reported half-step velocity is (j + F/2)/rho with j = 0."""
    sim.step()
    rho = sim.rho
    return 2.0 * rho[:, None] * sim.u.reshape(-1, 3)


def test_full_electric_force_matches_discrete_closed_form():
    """Eq. (force_el2) on a neutral fluid of uniform density: F = (eps - 1)/2
    grad|E|^2. With phi = A sin(kx) + B sin(ky + c) and a uniform applied
    field E0, the central-difference field is E_x = -A sin(k) cos(kx) + E0_x
    (E_y likewise), and the central difference of E_x^2 has the closed form
    -A^2 sin^2(k) sin(2k) sin(2kx)/2 + 2 A E0_x sin^2(k) sin(kx): the force
    must equal (eps - 1)/2 times it site by site. A wrong sign, a lost factor
    1/2 or eps in place of eps - 1 fails; the q E form gives no force here."""
    n, A, B, c, kap, r0 = 16, 0.02, -0.015, 0.3, 0.7, 1.5
    E0 = (3e-3, -2e-3, 5e-3)
    shape = (n, n, 4)
    N = n * n * 4
    x, y, z = [a.reshape(-1) for a in W._grid(shape)]
    k = 2 * np.pi / n
    phi = A * np.sin(k * x) + B * np.sin(k * y + c)
    eps = 1.0 + kap * r0
    s2 = np.sin(k) ** 2
    d_ex2 = -0.5 * A * A * s2 * np.sin(2 * k) * np.sin(2 * k * x) + 2 * A * E0[0] * s2 * np.sin(k * x)
    d_ey2 = -0.5 * B * B * s2 * np.sin(2 * k) * np.sin(2 * (k * y + c)) + 2 * B * E0[1] * s2 * np.sin(k * y + c)
    expect = np.stack([0.5 * (eps - 1.0) * d_ex2, 0.5 * (eps - 1.0) * d_ey2, np.zeros(N)], 1)
    for form in ("full", "qe"):
        cfg = W.base_params(shape=shape, G=0.0, Gw=0.0, charge_model="none", force_el=form,
                            eps_kappa=kap, E_ext=E0)
        sim = oracle.Sim(cfg, dict(mask=np.zeros(N, np.uint8), rho=np.full(N, r0)))
        sim.phi[:] = phi
        F = _force_from_step(sim)
        if form == "qe":
            assert np.abs(F).max() < 1e-18
            continue
        scale = np.abs(expect).max()
        assert scale > 1e-6
        assert np.abs(F - expect).max() <= 1e-12 * scale
        # the continuum force (eps-1)/2 d|E|^2/dx with E = -phi' + E0 agrees to O(k^2)
        ex = -A * k * np.cos(k * x) + E0[0]
        cont = 0.5 * (eps - 1.0) * 2 * ex * (A * k * k * np.sin(k * x))
        assert np.abs(F[:, 0] - cont).max() <= 0.2 * np.abs(cont).max()


def test_uniform_charge_in_uniform_field_gives_qE():
    """A uniform free charge q in a uniform applied field (neutralised
    background, so phi stays 0): the electric force of Eq. (force_el) is q E
    at every site and the total momentum rises by N q E in one step."""
    shape = (4, 6, 4)
    N = 96
    q0, E0 = 0.01, (0.3, -0.1, 0.2)
    cfg = W.base_params(shape=shape, G=0.0, Gw=0.0, charge_model="transport", E_ext=E0,
                        sigma_liq=0.02, sigma_gas=0.002)
    sim = oracle.Sim(cfg, dict(mask=np.zeros(N, np.uint8), rho=np.full(N, 1.3), q=np.full(N, q0)))
    r0, j0 = sim.moments()
    assert np.abs(j0).max() == 0.0
    F = _force_from_step(sim)
    assert np.abs(sim.phi).max() == 0.0
    assert np.allclose(sim.q, q0, rtol=1e-15, atol=0)
    expect = q0 * np.asarray(E0)
    assert np.abs(F - expect[None, :]).max() <= 1e-15 * np.abs(expect).max()
    r1, j1 = sim.moments()
    assert np.allclose(j1.sum(0), N * expect, rtol=1e-13, atol=0)


@pytest.mark.parametrize("face", ["harmonic", "arithmetic"])
def test_face_permittivity_series_law(face):
    """A slab layered along the electrode axis (eps varying with x only, no
    charge, electrodes at x = -1 and x = n): the flux J through every face is
    the same, so the potential drops by J times each face's resistance. With
    the harmonic face mean a face's resistance is the sum of its two
    half-cells' 1/(2 eps_i) + 1/(2 eps_j) (cells in series), with the
    arithmetic mean it is 1/((eps_i + eps_j)/2); an electrode face couples
    with the site's own eps. The solve must reproduce its own face law
    exactly and differ from the other one."""
    n = 12
    shape = (n, 2, 2)
    x = np.arange(n, dtype=float)
    kap, lo, hi = 1.0, 0.25, -0.6
    rho1 = 1.1 + 0.9 * np.sin(2 * np.pi * x / n) ** 2 + 0.3 * (x > 6)
    rho = np.tile(rho1, 4)
    eps = 1.0 + kap * rho1
    cfg = W.base_params(shape=shape, charge_model="xi", poisson_tol=1e-15, eps_kappa=kap, eps_face=face,
                        face_bc=["wall", "wall"] + ["periodic"] * 4,
                        phi_bc=["dirichlet", "dirichlet"] + ["periodic"] * 4,
                        phi_axis=0, phi_lo=lo, phi_hi=hi)
    phi, it, res = oracle.poisson_solve(cfg, np.zeros(4 * n, np.uint8), rho, np.zeros(4 * n))
    # series law: resistances of the n + 1 faces under each face mean
    def series(inner):
        Rf = np.concatenate([[1.0 / eps[0]], inner, [1.0 / eps[-1]]])
        return lo + (hi - lo) / Rf.sum() * np.cumsum(Rf)[:-1]
    laws = dict(harmonic=series(0.5 / eps[:-1] + 0.5 / eps[1:]),
                arithmetic=series(1.0 / (0.5 * (eps[:-1] + eps[1:]))))
    err = {k: np.abs(phi[:n] - v).max() / abs(hi - lo) for k, v in laws.items()}
    other = "arithmetic" if face == "harmonic" else "harmonic"
    assert err[face] <= 1e-12 and err[other] > 1e-4, err


def test_lagged_carreau_fixed_point_is_the_root():
    """The lagged reading of Eq. (strain2) (tau from the previous step's nu):
    for n = 1 it is nu0 at once; otherwise iterating it from nu0 converges to
    the root of Eq. (strain2) with Eq. (carreau), the reading the default
    step solves for, and a single application from nu0 differs from it."""
    cfg = W.base_params(nu0=1 / 6, nu_inf=1 / 60, n_carreau=0.5)
    cfg["lambda"] = 10.0
    rng = np.random.default_rng(41)
    for _ in range(20):
        Pn, a, rho = rng.uniform(5e-3, 5e-2), rng.uniform(1.8, 2.2), rng.uniform(0.2, 2.0)
        g_root, nu_root = oracle.carreau(cfg, Pn, a, rho)
        nu = cfg["nu0"]
        _, nu1 = oracle.carreau_lagged(cfg, Pn, a, rho, nu)
        for _ in range(400):
            gd, nu = oracle.carreau_lagged(cfg, Pn, a, rho, nu)
        assert nu == pytest.approx(nu_root, rel=1e-12)
        assert gd == pytest.approx(g_root, rel=1e-12)
        assert abs(nu1 - nu_root) > 1e-6 * nu_root
    newt = dict(cfg, n_carreau=1.0)
    assert oracle.carreau_lagged(newt, 2e-3, 2.0, 1.0, 0.05)[1] == newt["nu0"]
