"""Seeded synthetic workloads: parameter dictionaries and initial fields.

This module holds no step of the method. It only states the problems (lattice,
boundaries, material constants) and draws the seeded initial fields (density
profile with noise, initial charge, geometry mask, inlet profile). Both the
CUDA binding and the CPU oracle read these dictionaries; neither side's
arithmetic lives here.

Problems follow the setups of Lauricella et al. (arXiv:1612.05404), Sec. III:
liquid / vapour densities 2.0 / 0.16 at Shan-Chen coupling G = -5, psi scale
rho0 = 1, Newtonian viscosity 1/6, charged drop and electrified jet geometry.
The 3-D cases use the D3Q19 set.
"""
from __future__ import annotations

import math

import numpy as np

RHO_L = 2.0  # liquid density of the paper's runs (Sec. III A)
RHO_V = 0.16  # vapour density (Sec. III A)
FLUID, SOLID, INLET, OUTLET = 0, 1, 2, 3
SEED_BASE = 20161205

E0_SWEEP = (1e-4, 4e-4, 7e-4, 1e-3)


def base_params(**kw) -> dict:
    """Every parameter both sides read, with neutral defaults."""
    p = dict(
        dim=3, shape=(16, 16, 16),
        face_bc=["periodic"] * 6, phi_bc=["periodic"] * 6, phi_axis=2,
        charge_model="none", force_el="qe", neutralize=True,
        poisson_maxit=20000, poisson_fixed_sweeps=0, alpha_mode="entropic",
        phi_lo=0.0, phi_hi=0.0, phi_solid=0.0,
        nu0=1.0 / 6.0, nu_inf=1.0 / 6.0, n_carreau=1.0,
        G=-5.0, Gw=-5.0, rho0=1.0, eps_kappa=1.0,
        sigma_liq=0.0, sigma_gas=0.0, Dq=1e-3, E_ext=(0.0, 0.0, 0.0),
        Q_b=0.0, Q_s=0.0, K_d=1.0, xi_b=0.0, xi_s=0.0, theta_width=0.1,
        sor_omega=None, poisson_tol=1e-13, alpha_eq_tol=1e-8, eps_face="arithmetic", carreau_lagged=0,
        rho_in=RHO_L, rho_out=RHO_V,
        # CUDA-side choices (the oracle ignores them)
        precision="fp64", poisson_check_every=8, poisson_solver="sor", poisson_mg_cycles=50,
    )
    p["lambda"] = 0.0
    for k, v in kw.items():
        p[k] = v
    if p["sor_omega"] is None:
        nmax = max(p["shape"])
        p["sor_omega"] = 2.0 / (1.0 + math.sin(math.pi / nmax))
    return p


def reduced_precision(p: dict) -> dict:
    """Thresholds for FP32 arithmetic: the near-equilibrium alpha shortcut
    above the FP32 noise of Delta/f (about 3e-7), and a Poisson tolerance of
    1e-6 (the FP32 potential stops earlier at its rounding floor)."""
    if p["precision"] != "fp64":
        p["alpha_eq_tol"] = max(p["alpha_eq_tol"], 1e-5)
        p["poisson_tol"] = max(p["poisson_tol"], 1e-6)
    return p


def kappa_for_ratio(ratio: float, rho_l: float = RHO_L, rho_v: float = RHO_V) -> float:
    """kappa in eps = 1 + kappa rho such that eps(rho_l)/eps(rho_v) = ratio."""
    return (ratio - 1.0) / (rho_l - ratio * rho_v)


def _grid(shape):
    nx, ny, nz = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return x.astype(np.float64), y.astype(np.float64), z.astype(np.float64)


def drop_profile(shape, radius, center=None, width=5.0, dim=3):
    """tanh drop profile between RHO_L inside and RHO_V outside (x fastest)."""
    x, y, z = _grid(shape)
    nx, ny, nz = shape
    if center is None:
        center = ((nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0)
    r2 = (x - center[0]) ** 2 + (y - center[1]) ** 2
    if dim == 3:
        r2 = r2 + (z - center[2]) ** 2
    r = np.sqrt(r2)
    rho = 0.5 * (RHO_L + RHO_V) - 0.5 * (RHO_L - RHO_V) * np.tanh(2.0 * (r - radius) / width)
    return rho.reshape(-1)


def uniform_noise(n, amp, seed):
    return np.random.default_rng(seed).uniform(-amp, amp, size=n)


D3Q19_WEIGHTS = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def random_populations(n, amp, seed, rho_range=(0.16, 2.2)):
    """n synthetic D3Q19 sites, (19, n) FP64: f_p = w_p rho (1 + e_p) with rho
    uniform in rho_range and e_p uniform in [-amp, amp] (amp < 1 keeps every
    population positive). Inputs for the alpha root away from equilibrium:
    the relative departures e_p set the size of Delta_p / f_p."""
    rng = np.random.default_rng(seed)
    rho = rng.uniform(*rho_range, size=n)
    e = rng.uniform(-amp, amp, size=(19, n))
    return D3Q19_WEIGHTS[:, None] * rho[None, :] * (1.0 + e)


def charged_drop_at_rest(n=32, radius=8.0, precision="fp64", steps=500, seed=SEED_BASE + 1,
                         eps_ratio=2.0, sigma_ratio=10.0, Q=1e-3, noise=1e-4):
    """Charged drop at rest on an n^3 periodic D3Q19 lattice; the free charge is
    transported (advection-diffusion plus Ohmic relaxation)."""
    shape = (n, n, n)
    kappa = kappa_for_ratio(eps_ratio)
    eps_l = 1.0 + kappa * RHO_L
    sig_l = eps_l / 50.0
    cfg = base_params(shape=shape, charge_model="transport", eps_kappa=kappa,
                      sigma_liq=sig_l, sigma_gas=sig_l / sigma_ratio, Dq=1e-3,
                      precision=precision, poisson_tol=1e-13, poisson_solver="mg")
    reduced_precision(cfg)
    cfg["steps"] = steps
    N = n ** 3
    rho = drop_profile(shape, radius) + uniform_noise(N, noise, seed)
    inside = rho > 1.0
    q = np.where(inside, Q / max(int(inside.sum()), 1), 0.0)
    fields = dict(mask=np.zeros(N, np.uint8), rho=rho, q=q)
    return cfg, fields


# Box edges for batched droplets: every integer in [24, 96], odd ones
# included (periodic boxes of odd edge take the three-colour sweep and a
# multigrid hierarchy that coarsens odd extents).
BATCH_EDGES = tuple(range(24, 97))


def batched_droplet_params(n_boxes=512, seed=SEED_BASE + 5):
    """Per box (edge, E0, Carreau n), drawn from one seeded generator: edge
    uniform over BATCH_EDGES, E0 uniform in [0, 1e-3] (a uniform applied
    field along z), n uniform in [0.5, 1.0]."""
    rng = np.random.default_rng(seed)
    edges = rng.choice(BATCH_EDGES, size=n_boxes)
    E0 = rng.uniform(0.0, 1e-3, size=n_boxes)
    nc = rng.uniform(0.5, 1.0, size=n_boxes)
    return [(int(e), float(a), float(b)) for e, a, b in zip(edges, E0, nc)]


def batched_droplet(edge, E0, n_carreau, precision="fp32", seed=SEED_BASE + 5, Q=1e-3, noise=1e-4,
                    eps_ratio=2.0, sigma_ratio=10.0):
    """One box of the batched-droplets workload: periodic edge^3 lattice, drop
    of radius edge/4 at the centre, uniform applied field E0 along z, Carreau
    n_carreau with lambda = 10 and nu_inf = nu0/10, transported charge Q
    spread over rho > 1 (eps ratio 2, sigma ratio 10), density noise +-1e-4."""
    shape = (edge, edge, edge)
    kappa = kappa_for_ratio(eps_ratio)
    eps_l = 1.0 + kappa * RHO_L
    sig_l = eps_l / 50.0
    nu0 = 1.0 / 6.0
    cfg = base_params(shape=shape, charge_model="transport", eps_kappa=kappa,
                      sigma_liq=sig_l, sigma_gas=sig_l / sigma_ratio, Dq=1e-3,
                      E_ext=(0.0, 0.0, E0), nu0=nu0, nu_inf=nu0 / 10.0, n_carreau=n_carreau,
                      precision=precision, poisson_tol=1e-13, poisson_solver="mg")
    cfg["lambda"] = 10.0
    reduced_precision(cfg)
    N = edge ** 3
    rho = drop_profile(shape, edge / 4.0) + uniform_noise(N, noise, seed + edge)
    inside = rho > 1.0
    q = np.where(inside, Q / max(int(inside.sum()), 1), 0.0)
    return cfg, dict(rho=rho, q=q)


def drop_in_field(E0=1e-3, n=64, radius=12.0, precision="fp32", steps=5000,
                  seed=SEED_BASE + 2, eps_ratio=2.0, sigma_ratio=10.0, noise=1e-4,
                  n_carreau=0.6, lam=10.0):
    """Leaky-dielectric drop between electrodes: periodic in x, y; bounce-back
    walls carrying Dirichlet potentials on the z faces (E = E0 along z)."""
    shape = (n, n, n)
    kappa = kappa_for_ratio(eps_ratio)
    eps_l = 1.0 + kappa * RHO_L
    sig_l = eps_l / 50.0
    nu0 = 1.0 / 6.0
    cfg = base_params(
        shape=shape, charge_model="transport", eps_kappa=kappa,
        face_bc=["periodic", "periodic", "periodic", "periodic", "wall", "wall"],
        phi_bc=["periodic", "periodic", "periodic", "periodic", "dirichlet", "dirichlet"],
        phi_axis=2, phi_lo=0.0, phi_hi=-E0 * (n + 1),
        sigma_liq=sig_l, sigma_gas=sig_l / sigma_ratio, Dq=1e-3,
        nu0=nu0, nu_inf=nu0 / 10.0, n_carreau=n_carreau,
        precision=precision, poisson_tol=1e-13, poisson_solver="mg")
    reduced_precision(cfg)
    cfg["lambda"] = lam
    cfg["steps"] = steps
    cfg["E0"] = E0
    N = n ** 3
    rho = drop_profile(shape, radius) + uniform_noise(N, noise, seed)
    fields = dict(mask=np.zeros(N, np.uint8), rho=rho, q=np.zeros(N))
    return cfg, fields


def jet(shape=(128, 128, 512), nozzle_r=8, wall=2, nozzle_len=16, u_mean=0.02, E0=5e-4,
        precision="bf16", steps=20000, seed=SEED_BASE + 3, perturb=1e-3, adaptive_inlet=False):
    """Electrified jet (Sec. III B, extended to 3-D): a nozzle of inner radius
    nozzle_r along z injects liquid with a Poiseuille profile; outlet nodes at
    the far z plane are a vapour reservoir; lateral faces are walls; the
    potential drops linearly from 0 (nozzle side, nozzle conductor at 0) to
    -E0 (nz+1) (collector side). Charge is the non-conserved xi form. With
    adaptive_inlet the fluid sites inside the nozzle (r < nozzle_r,
    1 <= z < nozzle_len) are the region whose mean velocity rescales the inlet
    profile each step (fields["inlet_region"])."""
    nx, ny, nz = shape
    nu0 = 1.0 / 6.0
    cfg = base_params(
        shape=shape, charge_model="xi", xi_b=1e-4, xi_s=6e-2, K_d=1.0,
        face_bc=["wall"] * 6, phi_bc=["dirichlet"] * 6, phi_axis=2,
        phi_lo=0.0, phi_hi=-E0 * (nz + 1), phi_solid=0.0,
        nu0=nu0, nu_inf=nu0 / 10.0, n_carreau=0.5, eps_kappa=1.0,
        precision=precision, poisson_tol=1e-13)
    reduced_precision(cfg)
    cfg["lambda"] = 20.0
    cfg["steps"] = steps
    x, y, z = _grid(shape)
    cx, cy = (nx - 1) / 2.0, (ny - 1) / 2.0
    r = np.sqrt((x - cx) ** 2 + (y - cy) ** 2).reshape(-1)
    zf = z.reshape(-1)
    mask = np.zeros(nx * ny * nz, np.uint8)
    mask[(r >= nozzle_r) & (r < nozzle_r + wall) & (zf < nozzle_len)] = SOLID
    inlet = (r < nozzle_r) & (zf == 0)
    mask[inlet] = INLET
    mask[zf == nz - 1] = OUTLET
    rho = np.full(nx * ny * nz, RHO_V)
    rho[(r < nozzle_r) & (zf < nozzle_len)] = RHO_L
    # a drop just outside the nozzle, as in the paper's initial state
    d = np.sqrt((x.reshape(-1) - cx) ** 2 + (y.reshape(-1) - cy) ** 2 + (zf - nozzle_len) ** 2)
    rho = np.maximum(rho, 0.5 * (RHO_L + RHO_V) - 0.5 * (RHO_L - RHO_V) * np.tanh(2.0 * (d - nozzle_r) / 5.0))
    rho[mask == SOLID] = 0.0
    u_in = np.zeros((nx * ny * nz, 3))
    prof = 2.0 * u_mean * (1.0 - (r / nozzle_r) ** 2)
    pert = uniform_noise(nx * ny * nz, perturb, seed)
    u_in[inlet, 2] = prof[inlet] + pert[inlet]
    fields = dict(mask=mask, rho=rho, q=np.zeros(nx * ny * nz), u_in=u_in)
    if adaptive_inlet:
        fields["inlet_region"] = ((r < nozzle_r) & (zf >= 1) & (zf < nozzle_len) & (mask == FLUID)).astype(np.uint8)
    return cfg, fields


def paper_drop_2d(n=320, radius=40.0, Q=2.13, qs_over_qb=10.0, steps=1000,
                  seed=SEED_BASE + 6, noise=0.0):
    """The paper's 2-D charged drop at rest (Sec. III A): D2Q9, periodic n x n,
    R = 40, G = -5, Q = 2.13 with Q_s/Q_b = 10, K_d = 1, nu = 1/6, eps = 1 + rho."""
    shape = (n, n, 1)
    Q_b = Q / (1.0 + qs_over_qb)
    cfg = base_params(dim=2, shape=shape, charge_model="conserved", Q_b=Q_b,
                      Q_s=Q - Q_b, K_d=1.0, eps_kappa=1.0, phi_axis=0)
    cfg["steps"] = steps
    rho = drop_profile(shape, radius, dim=2)
    if noise:
        rho = rho + uniform_noise(n * n, noise, seed)
    fields = dict(mask=np.zeros(n * n, np.uint8), rho=rho)
    return cfg, fields


JET2D_CASES = {  # Sec. III B: Newtonian, then Carreau with flow index 0.75 and 0.5
    "a": dict(n_carreau=1.0, nu_inf=1.0 / 6.0, lam=0.0),
    "b": dict(n_carreau=0.75, nu_inf=1e-3, lam=1000.0),
    "c": dict(n_carreau=0.5, nu_inf=1e-3, lam=1000.0),
}


def jet_2d(n=320, D=40, case="a", nozzle_len=40, wall=5, u_mean=0.02, E0=0.1,
           precision="fp64", steps=20000, seed=SEED_BASE + 7, perturb=0.0,
           rho_in=RHO_L, rho_out=RHO_V):
    """The paper's 2-D electrified jet (Sec. III B) on D2Q9: an n x n lattice,
    x along the jet. A nozzle of inner diameter D on the left (bore
    |y - c| < D/2, walls `wall` sites thick, x < nozzle_len; a conductor at
    the potential of the left side) holds the inlet nodes at x = 0; outlet
    nodes at x = n - 1 are a vapour reservoir (rho 0.16); every face is a
    bounce-back wall. The potential is 0 on the left ghost plane and
    -E0 (n + 1) on the right one, linear along the upper and lower sides (a
    field E0 along x); the charge is the xi form (1e-4, 6e-2), neutralised;
    G = Gw = -5, eps = 1 + rho. The inlet profile is Poiseuille, rescaled
    each step to the mean velocity measured inside the nozzle
    (fields["inlet_region"]). Liquid fills the nozzle with a drop just
    outside it. `case` picks the rheology (JET2D_CASES). rho_in / rho_out:
    the densities held by the inlet and outlet nodes (the paper's printed
    2.0 / 0.16 by default)."""
    rh = JET2D_CASES[case]
    shape = (n, n, 1)
    nu0 = 1.0 / 6.0
    cfg = base_params(
        dim=2, shape=shape, charge_model="xi", xi_b=1e-4, xi_s=6e-2, K_d=1.0,
        face_bc=["wall"] * 6, phi_bc=["dirichlet"] * 4 + ["neumann"] * 2, phi_axis=0,
        phi_lo=0.0, phi_hi=-E0 * (n + 1), phi_solid=0.0,
        nu0=nu0, nu_inf=rh["nu_inf"], n_carreau=rh["n_carreau"], eps_kappa=1.0,
        precision=precision, poisson_tol=1e-13, rho_in=rho_in, rho_out=rho_out)
    reduced_precision(cfg)
    cfg["lambda"] = rh["lam"]
    cfg["steps"] = steps
    N = n * n
    x = np.tile(np.arange(n), n).astype(float)
    y = np.repeat(np.arange(n), n).astype(float)
    yc = (n - 1) / 2.0
    a0 = D / 2.0
    ry = np.abs(y - yc)
    mask = np.zeros(N, np.uint8)
    mask[(ry >= a0) & (ry < a0 + wall) & (x < nozzle_len)] = SOLID
    inlet = (ry < a0) & (x == 0)
    mask[inlet] = INLET
    mask[x == n - 1] = OUTLET
    rho = np.full(N, RHO_V)
    rho[(ry < a0) & (x < nozzle_len)] = RHO_L
    d = np.sqrt((x - nozzle_len) ** 2 + (y - yc) ** 2)
    rho = np.maximum(rho, 0.5 * (RHO_L + RHO_V) - 0.5 * (RHO_L - RHO_V) * np.tanh(2.0 * (d - a0) / 5.0))
    rho[mask == SOLID] = 0.0
    u_in = np.zeros((N, 3))
    prof = 1.5 * u_mean * (1.0 - (ry / a0) ** 2)  # 2-D Poiseuille: peak 3/2 of the mean
    u_in[inlet, 0] = prof[inlet]
    if perturb:
        u_in[inlet, 0] += uniform_noise(N, perturb, seed)[inlet]
    fields = dict(mask=mask, rho=rho, q=np.zeros(N), u_in=u_in,
                  inlet_region=((ry < a0) & (x >= 1) & (x < nozzle_len) & (mask == FLUID)).astype(np.uint8))
    return cfg, fields


def as_float64_fields(fields: dict) -> dict:
    out = {}
    for k, v in fields.items():
        out[k] = np.ascontiguousarray(v, dtype=np.uint8 if k == "mask" else np.float64)
    return out
