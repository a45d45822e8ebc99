"""The paper's own 2-D method on the GPU: the D2Q9 set (Sec. II) through the
C ABI against the FP64 oracle's 2-D path, element by element on seeded
inputs (FP64 to 1e-12 relative, FP32 within the tolerances of the 3-D
tests), and the paper's 2-D numbers (Sec. III A) from GPU runs at its size."""
import numpy as np
import pytest

import oracle
from paper_1612_05404_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1612_05404_gb300 import build, elbm
    build.build()
    return elbm


def rel_inf(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _rho_u(rho, u):
    return u.reshape(-1, 3) * rho[:, None]


def _tight(cfg):
    cfg.update(poisson_solver="sor", poisson_check_every=1, poisson_tol=1e-13, precision="fp64",
               store_macro=1)
    return cfg


def _fields(sim):
    """The compared fields of a GPU or an oracle run (rho_u: momentum density)."""
    get = sim.get if hasattr(sim, "get") else (lambda k: getattr(sim, k))
    return dict(f=get("f"), rho=get("rho"), rho_u=_rho_u(get("rho"), get("u")), nu=get("nu"),
                phi=get("phi"), q=get("q"), alpha=get("alpha"))


def field_errors(a, b):
    """L-inf difference of each field relative to its largest magnitude,
    except the momentum density j = sum_p f_p c_p: a cancelling sum (a drop
    at rest has |j| << rho) whose error is bounded by that of its terms,
    sum_p f_p |c_pa| <= rho, so it is taken relative to the largest density."""
    out = {k: rel_inf(a[k], b[k]) for k in a if k != "rho_u"}
    out["rho_u"] = float(np.abs(a["rho_u"] - b["rho_u"]).max() / np.abs(b["rho"]).max())
    return out


def oracle_spread(cfg, fl, steps, seeds=(11, 12, 13, 14)):
    """The oracle's own sensitivity to rounding: the same run from the initial
    density perturbed by 1e-15 relative (a few units in the last place),
    the largest change of each field (field_errors) over the perturbations.
    Where the method is ill-conditioned (the xi charge's (K/K_d)^(1/4) at a
    flat interface, whose K is rounding noise; an alpha root near a branch)
    no two summation orders agree to 1e-12, and a parity bound below this
    spread would test the order of the sums. Returns the unperturbed run
    and the spread."""
    ref = oracle.Sim(cfg, fl)
    ref.step(steps)
    r = _fields(ref)
    out = {}
    for sd in seeds:
        rng = np.random.default_rng(sd)
        f2 = dict(fl, rho=np.asarray(fl["rho"]) * (1.0 + 1e-15 * rng.standard_normal(np.size(fl["rho"]))))
        o = oracle.Sim(cfg, f2)
        o.step(steps)
        for k, v in field_errors(_fields(o), r).items():
            out[k] = max(out.get(k, 0.0), v)
    return ref, out


def compare_fp64(g, o, cfg, tol=1e-12, tol_nu=1e-12, spread=None):
    """Each field (field_errors) within tol, the viscosity within tol_nu
    (where the Carreau law is steep, lambda gdot ~ 1, it inherits the alpha
    root's tolerance through A = Pi alpha / (rho c_s^2)), or within twice
    the oracle's own spread where one is given: the GPU's summation order is
    a rounding perturbation of another kind than the spread's input noise."""
    gf, of = _fields(g), _fields(o)
    keys = ["f", "rho", "rho_u", "nu"] + (["phi", "q"] if cfg["charge_model"] != "none" else [])
    out = {k: v for k, v in field_errors(gf, of).items() if k in keys}
    sp = spread or {}
    bad = {k: v for k, v in out.items() if not v <= max(tol_nu if k == "nu" else tol, 2.0 * sp.get(k, 0.0))}
    assert not bad, (bad, out, sp)
    return out


def test_d2q9_streaming_roundtrip_bit_exact(E):
    """Populations given explicitly in the D2Q9 order come back unchanged
    from the device layout: an exact permutation with walls, solids, inlet
    and outlet nodes (links from inlet/outlet nodes carry their equilibria)."""
    shape = (10, 8, 1)
    nx, ny, _ = shape
    N = nx * ny
    cfg = W.base_params(dim=2, shape=shape, phi_axis=0,
                        face_bc=["periodic"] * 2 + ["wall"] * 4,
                        phi_bc=["periodic"] * 2 + ["neumann"] * 4)
    mask = np.zeros(N, np.uint8)
    mask[[23, 24, 51]] = W.SOLID
    mask[np.arange(ny) * nx] = W.INLET
    mask[np.arange(ny) * nx + nx - 1] = W.OUTLET
    rng = np.random.default_rng(200)
    f0 = rng.uniform(0.01, 0.2, 9 * N)
    f0.reshape(9, N)[:, mask != 0] = 0.0
    u_in = np.zeros((N, 3))
    u_in[mask == W.INLET, 0] = 0.02
    ref = oracle.Sim(cfg, dict(mask=mask, rho=np.ones(N), f=f0, u_in=u_in)).f.reshape(9, N)
    c, w = E.velocity_set(2)
    xs, ys = np.arange(N) % nx, np.arange(N) // nx
    io_link = np.zeros((9, N), bool)
    for p in range(9):
        sx, sy = (xs - c[p, 0]) % nx, ys - c[p, 1]
        ok = (sy >= 0) & (sy < ny)
        src = sx + nx * np.clip(sy, 0, ny - 1)
        io_link[p] = ok & ((mask[src] == W.INLET) | (mask[src] == W.OUTLET))
    fl = np.broadcast_to(mask == 0, (9, N))
    perm, io = fl & ~io_link, fl & io_link
    for prec in ("fp64", "fp32"):
        cfg["precision"] = prec
        W.reduced_precision(cfg)
        g = E.Sim(cfg, dict(mask=mask, rho=np.ones(N), f=f0, u_in=u_in))
        out = g.get("f").reshape(9, N)
        if prec == "fp64":
            assert np.array_equal(out[perm], ref[perm])
            assert np.allclose(out[io], ref[io], rtol=4e-16, atol=0)
        else:
            expect = (ref - w[:, None]).astype(np.float32).astype(np.float64) + w[:, None]
            assert np.array_equal(out[perm], expect[perm])
            assert np.allclose(out[io], ref[io], rtol=2e-7, atol=0)
        g.close()


def test_d2q9_fp64_paper_drop_conserved_charge(E):
    """The paper's charged drop at rest (Eq. surface-q2, Q = 2.13, Q_s/Q_b =
    10, eps = 1 + rho) on a 40^2 lattice with density noise: every field
    and alpha against the oracle after 4 steps; alpha to 1e-9 or the
    oracle's own spread under rounding-level input noise (measured: GPU
    2.7e-9, spread 1.6e-8; its effect on f stays below 1e-12)."""
    cfg, fl = W.paper_drop_2d(n=40, radius=8.0, noise=1e-3)
    _tight(cfg)
    g = E.Sim(cfg, fl)
    g.step(4)
    o, sp = oracle_spread(cfg, fl, 4)
    compare_fp64(g, o, cfg)
    assert rel_inf(g.get("alpha"), o.alpha) <= max(1e-9, 2.0 * sp["alpha"]), sp


def test_d2q9_fp64_drop_in_applied_field(E):
    """The drop in a uniform applied field (Sec. III A, E_ext = 0.1 along x),
    with the FULL electric force Eq. (force_el2) and a Carreau liquid
    (lambda = 1000: the viscosity held to the alpha root's 1e-9, measured
    3.8e-10)."""
    cfg, fl = W.paper_drop_2d(n=36, radius=7.0, noise=1e-3)
    cfg.update(E_ext=(0.1, 0.0, 0.0), force_el="full", n_carreau=0.5, nu_inf=1e-3)
    cfg["lambda"] = 1000.0
    _tight(cfg)
    g = E.Sim(cfg, fl)
    g.step(4)
    o = oracle.Sim(cfg, fl)
    o.step(4)
    compare_fp64(g, o, cfg, tol_nu=1e-9)
    assert g.get("nu").min() < cfg["nu0"]  # the Carreau branch ran


@pytest.mark.parametrize("case", ["a", "b", "c"])
def test_d2q9_fp64_jet(E, case):
    """The paper's 2-D jet (Sec. III B) scaled to 48^2: nozzle conductor,
    inlet and outlet nodes, walls, electrodes with the linear side profile,
    the xi charge, the adaptive Poiseuille inlet and the three rheologies
    (the Carreau cases' viscosity to the alpha root's 1e-9). The inlet scale
    is the nozzle's mean velocity over the initial profile's mean m0 (0.02),
    so it carries the velocities' error times max|u| / m0: held to
    10 tol max|u| / m0 (measured 7.6e-12 at max|u| ~ 0.1). The fields to
    1e-12 or the oracle's own spread under rounding-level input noise: the
    nozzle's flat interfaces make the xi charge ill-conditioned (spread
    ~2e-8 in f after 3 steps; the GPU measured 3e-9)."""
    cfg, fl = W.jet_2d(n=48, D=12, nozzle_len=10, wall=2, case=case)
    _tight(cfg)
    g = E.Sim(cfg, fl)
    _, sp = oracle_spread(cfg, fl, 3)
    o = oracle.Sim(cfg, fl)
    inlet = o.mask == oracle.INLET
    u0 = fl["u_in"][inlet, 0]
    m0 = float(u0.mean())
    for t in range(3):
        g.step(1)
        o.step(1)
        scale_o = float(np.mean(o.u_in.reshape(-1, 3)[inlet, 0] / u0))
        umax = float(np.abs(o.u).max())
        assert abs(g.diag()["inlet_scale"] - scale_o) <= 1e-11 * umax / m0, (t, scale_o, umax)
    compare_fp64(g, o, cfg, tol_nu=1e-12 if case == "a" else 1e-9, spread=sp)
    assert abs(scale_o - 1.0) > 1e-2  # the inlet followed the nozzle


@pytest.mark.parametrize("aprec", ["fp64", "fp32"])
def test_d2q9_fp32_jet_two_steps(E, aprec):
    """FP32 populations on the 2-D jet (case c: Carreau n = 0.5, the FP64 or
    the guarded FP32 root) against the FP64 oracle over two steps, relative
    L2 over the fluid: density, momentum, potential and charge within 1e-5
    (measured up to 8.9e-6, the xi charge's (K/K_d)^(1/4) being steep at
    small K). As in the 3-D jet tests alpha is not compared site by site:
    at the start the inlet scale is a small difference of opposite flows
    (about 0.004), which FP32 resolves to ~1e-2 of itself, and the roots
    next to the inlet follow it (2 to 30e-5 relative L2); the FP32 root's
    own criterion, the H-error, is held by the test below."""
    cfg, fl = W.jet_2d(n=48, D=12, nozzle_len=10, wall=2, case="c", precision="fp32")
    cfg.update(store_macro=1, alpha_precision=aprec)
    g = E.Sim(cfg, fl)
    o = oracle.Sim(dict(cfg, poisson_tol=1e-13), fl)
    for t in range(2):
        g.step(1)
        o.step(1)
        fluid = o.mask == oracle.FLUID
        errs = dict(rho=rel_l2(g.get("rho")[fluid], o.rho[fluid]), phi=rel_l2(g.get("phi"), o.phi),
                    q=rel_l2(g.get("q"), o.q),
                    rho_u=rel_l2(_rho_u(g.get("rho"), g.get("u"))[fluid], _rho_u(o.rho, o.u)[fluid]))
        assert max(errs.values()) < 1e-5, (t, errs)


def test_d2q9_fp32_paper_drop_h_error(E):
    """The guarded FP32 alpha root on the paper's drop in a field (60^2,
    E_ext = 0.1, 40 steps): every step's max H-error |h(alpha)|/rho at or
    below 1e-10 against the exact equation of the stored populations, no
    guard failure and no non-finite value; density and charge against the
    FP64 oracle within 1e-5 relative L2 after the 40 steps (the potential,
    periodic and neutralised, stops at the FP32 solve's rounding floor)."""
    cfg, fl = W.paper_drop_2d(n=60, radius=12.0, noise=1e-3)
    cfg.update(E_ext=(0.1, 0.0, 0.0), precision="fp32", alpha_precision="fp32", store_macro=1)
    W.reduced_precision(cfg)
    g = E.Sim(cfg, fl)
    for t in range(40):
        g.step(1)
        d = g.diag()
        assert d["max_h_error"] <= 1e-10, (t, d["max_h_error"])
        assert d["n_guard_failed"] == 0 and d["n_nonfinite"] == 0, (t, d)
    o = oracle.Sim(dict(cfg, poisson_tol=1e-13), fl)
    o.step(40)
    assert rel_l2(g.get("rho"), o.rho) < 1e-5
    assert rel_l2(g.get("q"), o.q) < 1e-5


def _eos(rho, G):
    """Shan-Chen pressure p = rho c_s^2 + G c_s^2 psi^2 / 2, psi = 1 - exp(-rho)."""
    return rho / 3.0 + G / 6.0 * (1.0 - np.exp(-rho)) ** 2


def test_d2q9_laplace_law_surface_tension(E, paper):
    """Drops at G = -5 with the entropic root (FP64, the drops and step
    count of the oracle's BGK pin): Delta p = sigma / R with sigma the same
    for both radii within 2 % and within 10 % of the paper's 5.8e-2
    (Sec. III A)."""
    sig = []
    for n, R in ((40, 9.0), (48, 13.0)):
        cfg = W.base_params(dim=2, shape=(n, n, 1), phi_axis=0)
        g = E.Sim(cfg, dict(mask=np.zeros(n * n, np.uint8), rho=W.drop_profile((n, n, 1), R, dim=2)))
        g.step(2500)
        r = g.get("rho").reshape(n, n)
        rin, rout = r[n // 2, n // 2], r[0, 0]
        Req = np.sqrt((r - rout).sum() / (rin - rout) / np.pi)
        sig.append((_eos(rin, -5.0) - _eos(rout, -5.0)) * Req)
        g.close()
    assert sig[0] == pytest.approx(sig[1], rel=0.02)
    assert float(np.mean(sig)) == pytest.approx(paper["sigma"]["value"], rel=0.10)


def test_d2q9_paper_charged_drop_at_rest_full_size(E, paper):
    """The paper's charged drop at rest at its own size (320^2, R = 40,
    Q = 2.13, Q_s/Q_b = 10, eps = 1 + rho) after its 1000 steps, FP64:
    the free charge still sums to Q; outside the drop |E| follows Gauss's
    law |E| = Q_enc/(2 pi r eps_V) within 2 %, and the paper's boundary
    value 3.5e-3 lies within the range of |E| across the interface."""
    cfg, fl = W.paper_drop_2d()
    cfg.update(poisson_tol=1e-10, store_macro=1)
    n = 320
    g = E.Sim(cfg, fl)
    g.step(1000)
    d = g.diag()
    Q = paper["Q_total"]["value"]
    assert d["n_nonfinite"] == 0
    rho, q, phi = g.get("rho"), g.get("q"), g.get("phi")
    assert abs(q.sum() - Q) <= 1e-9 * Q
    Em = np.sqrt((oracle.efield(cfg, fl["mask"], phi) ** 2).sum(1))
    x = np.arange(n) - 159.5
    dist = np.sqrt(x[None, :] ** 2 + x[:, None] ** 2).reshape(-1)
    eps_v = 1.0 + rho[0]
    for r in (60.0, 80.0):
        sel = np.abs(dist - r) < 0.5
        q_enc = Q * (1.0 - np.pi * r ** 2 / n ** 2)
        assert Em[sel].mean() == pytest.approx(q_enc / (2 * np.pi * r * eps_v), rel=0.02)
    band = (dist > 37.0) & (dist < 45.0)
    Eb = paper["E_boundary"]["value"]
    assert Em[band].min() < Eb < Em[band].max()
    g.close()


def _aspect(rho, n, rho_v=0.16):
    """sqrt(I_xx / I_yy) of the liquid's excess density (x: the field's axis)."""
    w = np.clip(rho.reshape(n, n) - rho_v, 0.0, None)
    y, x = np.mgrid[0:n, 0:n]
    m = w.sum()
    cx, cy = (w * x).sum() / m, (w * y).sum() / m
    return float(np.sqrt((w * (x - cx) ** 2).sum() / (w * (y - cy) ** 2).sum()))


def test_d2q9_paper_drop_in_applied_field_full_size(E, paper):
    """The paper's charged drop in an applied field at its own size (320^2,
    R = 40, E_ext = 0.1 and 0.5 along x, t = 1250, FP64; Sec. III A), here
    started from the initial tanh profile (the paper starts from the drop
    equilibrated at rest): the drop stays finite and stretches along the
    field, more at 0.5 than at 0.1, and its interface curvature K (the
    oracle's K of the GPU's density, maximum over 0.6 < rho < 1.6) grows
    from about 1/R. Measured: aspect 1.015 and 1.41, K_max 0.028 and 0.113;
    the paper prints K_max = 5.17e-2 at 0.5 for its protocol and measure
    (held here only as an order of magnitude)."""
    n = 320
    res = {}
    for e_ext in (0.1, 0.5):
        cfg, fl = W.paper_drop_2d()
        cfg.update(E_ext=(e_ext, 0.0, 0.0), poisson_tol=1e-10, store_macro=1)
        g = E.Sim(cfg, fl)
        for _ in range(5):
            g.step(250)
        assert g.diag()["n_nonfinite"] == 0
        rho = g.get("rho")
        _, K, _ = oracle.charge_field(cfg, fl["mask"], rho)
        band = (rho > 0.6) & (rho < 1.6)
        res[e_ext] = (_aspect(rho, n), float(K[band].max()))
        g.close()
    (a1, k1), (a5, k5) = res[0.1], res[0.5]
    assert 1.0 < a1 < 1.05 and 1.2 < a5 < 1.6, res
    assert 0.9 / 40.0 < k1 < 1.25 / 40.0, res
    assert k5 > 2.0 * k1, res
    kp = paper["K_max"]["value"]
    assert 0.5 * kp < k5 < 4.0 * kp, res
