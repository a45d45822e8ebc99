"""Pins of the oracle's lattice layer: velocity sets, Eq. (2) equilibrium,
streaming as an exact permutation, BGK limit, conservation."""
import numpy as np
import pytest

import oracle
from paper_1612_05404_gb300 import workloads as W


@pytest.mark.parametrize("dim", [2, 3])
def test_velocity_set_isotropy(dim, paper):
    c, w, cs2 = oracle.lattice(dim)
    assert cs2 == pytest.approx(paper["cs2"]["value"], rel=1e-15)
    if dim == 2:
        # weights printed after Eq. (2)
        w0, w1, w2 = paper["weights_d2q9"]["values"]
        speed2 = (c ** 2).sum(1)
        assert np.allclose(w[speed2 == 0], w0) and np.allclose(w[speed2 == 1], w1)
        assert np.allclose(w[speed2 == 2], w2)
    cf = c.astype(float)
    d = np.eye(3)[:dim, :dim]
    cf = cf[:, :dim]
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    assert np.abs(np.einsum("p,pa->a", w, cf)).max() < 1e-15
    assert np.allclose(np.einsum("p,pa,pb->ab", w, cf, cf), cs2 * d, atol=1e-15)
    assert np.abs(np.einsum("p,pa,pb,pc->abc", w, cf, cf, cf)).max() < 1e-15
    m4 = np.einsum("p,pa,pb,pc,pd->abcd", w, cf, cf, cf, cf)
    iso = cs2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                      + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(m4, iso, atol=1e-15)
    # every velocity has its opposite
    for v in c:
        assert any((c == -v).all(1))


@pytest.mark.parametrize("dim", [2, 3])
def test_feq_moments(dim):
    """Eq. (2) reproduces rho, rho u and rho c_s^2 I + rho u u exactly."""
    c, w, cs2 = oracle.lattice(dim)
    rng = np.random.default_rng(1)
    for _ in range(20):
        rho = rng.uniform(0.1, 2.5)
        u = np.zeros(3)
        u[:dim] = rng.uniform(-0.2, 0.2, dim)
        fe = oracle.feq(dim, rho, u)
        cf = c.astype(float)
        assert fe.sum() == pytest.approx(rho, rel=1e-14)
        assert np.allclose(fe @ cf, rho * u, atol=1e-15)
        P = np.einsum("p,pa,pb->ab", fe, cf, cf)[:dim, :dim]
        expect = rho * cs2 * np.eye(dim) + rho * np.outer(u[:dim], u[:dim])
        assert np.allclose(P, expect, atol=1e-14)


def _geometry_cfg():
    cfg = W.base_params(shape=(6, 4, 5),
                        face_bc=["periodic", "periodic", "wall", "wall", "periodic", "periodic"],
                        phi_bc=["periodic", "periodic", "neumann", "neumann", "periodic", "periodic"])
    mask = np.zeros(6 * 4 * 5, np.uint8)
    mask[[7, 30, 55, 101]] = oracle.SOLID
    return cfg, mask


def test_streaming_is_a_permutation():
    """Streaming moves every fluid population exactly once (halfway
    bounce-back at walls and solids, periodic wrap elsewhere): a bijection on
    the fluid populations, bit-exact."""
    cfg, mask = _geometry_cfg()
    N = mask.size
    rng = np.random.default_rng(2)
    fs = rng.uniform(0.0, 1.0, 19 * N)
    fs.reshape(19, N)[:, mask != 0] = 0.0
    out, _ = oracle.stream(cfg, mask, fs)
    fl = mask == 0
    a = np.sort(fs.reshape(19, N)[:, fl].ravel())
    b = np.sort(out.reshape(19, N)[:, fl].ravel())
    assert np.array_equal(a, b)
    # D3Q7 charge populations too
    gs = rng.uniform(0.0, 1.0, 7 * N)
    gs.reshape(7, N)[:, mask != 0] = 0.0
    _, gout = oracle.stream(cfg, mask, fs, gs)
    assert np.array_equal(np.sort(gs.reshape(7, N)[:, fl].ravel()),
                          np.sort(gout.reshape(7, N)[:, fl].ravel()))


def test_single_population_lands_at_r_plus_c():
    """Brute force: a lone population at (r, p) arrives at r + c_p, or at
    (r, opp(p)) when r + c_p is a wall node."""
    cfg, mask = _geometry_cfg()
    nx, ny, nz = cfg["shape"]
    N = nx * ny * nz
    c, _, _ = oracle.lattice(3)
    rng = np.random.default_rng(3)
    fluid = np.flatnonzero(mask == 0)
    for _ in range(60):
        s = int(rng.choice(fluid))
        p = int(rng.integers(0, 19))
        fs = np.zeros(19 * N)
        fs[p * N + s] = 1.0
        out, _ = oracle.stream(cfg, mask, fs)
        x, y, z = s % nx, (s // nx) % ny, s // (nx * ny)
        tx, ty, tz = x + c[p, 0], y + c[p, 1], z + c[p, 2]
        if ty < 0 or ty >= ny:
            target = (int(np.flatnonzero((c == -c[p]).all(1))[0]), s)
        else:
            t = (tx % nx) + nx * (ty + ny * (tz % nz))
            if mask[t] == oracle.SOLID:
                target = (int(np.flatnonzero((c == -c[p]).all(1))[0]), s)
            else:
                target = (p, t)
        nz_idx = np.flatnonzero(out)
        assert nz_idx.tolist() == [target[0] * N + target[1]]


def test_bgk_limit_matches_textbook_bgk():
    """alpha forced to 2 reduces Eq. (lattice-b) to BGK with
    tau = nu/c_s^2 + 1/2 (Eq. beta), streamed by c: compared with a textbook
    numpy BGK with np.roll streaming on a periodic D2Q9 lattice."""
    nx, ny = 8, 6
    cfg = W.base_params(dim=2, shape=(nx, ny, 1), alpha_mode="bgk", G=0.0, Gw=0.0,
                        nu0=0.1, nu_inf=0.1, phi_axis=0)
    rng = np.random.default_rng(4)
    rho0 = 1.0 + 0.05 * rng.standard_normal(nx * ny)
    sim = oracle.Sim(cfg, dict(mask=np.zeros(nx * ny, np.uint8), rho=rho0))
    c, w, cs2 = oracle.lattice(2)
    f = sim.f.reshape(9, ny, nx) * (1.0 + 0.02 * rng.standard_normal((9, ny, nx)))
    sim.f[:] = f.reshape(-1)
    tau = 0.1 / cs2 + 0.5
    for _ in range(3):
        rho = f.sum(0)
        ux = (f * c[:, 0, None, None]).sum(0) / rho
        uy = (f * c[:, 1, None, None]).sum(0) / rho
        fe = np.empty_like(f)
        for p in range(9):
            cu = 3.0 * (c[p, 0] * ux + c[p, 1] * uy)
            fe[p] = w[p] * rho * (1 + cu + 0.5 * cu ** 2 - 1.5 * (ux ** 2 + uy ** 2))
        fs = f - (f - fe) / tau
        f = np.stack([np.roll(np.roll(fs[p], c[p, 0], axis=1), c[p, 1], axis=0) for p in range(9)])
        sim.step()
    assert np.allclose(sim.f.reshape(9, ny, nx), f, rtol=1e-13, atol=1e-15)


def test_mass_and_charge_conserved_periodic():
    """Sum rho and sum q are invariants of the periodic step (collision
    conserves mass, Eq. add adds none, transport source integrates to zero)."""
    cfg, fields = W.charged_drop_at_rest(n=12, radius=3.5)
    sim = oracle.Sim(cfg, fields)
    m0 = sim.moments()[0].sum()
    q0 = sim.g.reshape(7, -1).sum()
    for _ in range(3):
        sim.step()
    assert sim.moments()[0].sum() == pytest.approx(m0, rel=1e-13)
    assert sim.g.reshape(7, -1).sum() == pytest.approx(q0, rel=1e-12)


def test_mass_conserved_with_walls():
    cfg, fields = W.drop_in_field(E0=1e-3, n=10, radius=3.0, precision="fp64")
    sim = oracle.Sim(cfg, fields)
    m0 = sim.moments()[0].sum()
    for _ in range(3):
        sim.step()
    assert sim.moments()[0].sum() == pytest.approx(m0, rel=1e-13)


def test_inlet_and_outlet_populations():
    """Populations streaming out of an inlet node are its equilibrium
    f^eq(rho_in, u_in); out of an outlet node, f^eq(rho_out, 0)."""
    shape = (4, 4, 6)
    N = 96
    cfg = W.base_params(shape=shape, face_bc=["periodic"] * 4 + ["wall", "wall"],
                        phi_bc=["periodic"] * 4 + ["dirichlet", "dirichlet"],
                        rho_in=1.9, rho_out=0.2)
    mask = np.zeros(N, np.uint8)
    mask[:16] = oracle.INLET       # z = 0 plane
    mask[80:] = oracle.OUTLET      # z = 5 plane
    u_in = np.zeros((N, 3))
    u_in[:16, 2] = np.linspace(0.01, 0.03, 16)
    fs = np.random.default_rng(5).uniform(0, 1, 19 * N)
    out, _ = oracle.stream(cfg, mask, fs, u_in=u_in)
    c, _, _ = oracle.lattice(3)
    out = out.reshape(19, N)
    for s in range(16, 32):  # z = 1 plane: links with c_z = +1 come from the inlet
        for p in np.flatnonzero(c[:, 2] == 1):
            srcp = (s % 4 - c[p, 0]) % 4 + 4 * ((s // 4 % 4 - c[p, 1]) % 4)
            fe = oracle.feq(3, 1.9, u_in[srcp])
            assert out[p, s] == fe[p]
    fo = oracle.feq(3, 0.2, [0, 0, 0])
    for s in range(64, 80):  # z = 4 plane: links with c_z = -1 come from the outlet
        for p in np.flatnonzero(c[:, 2] == -1):
            assert out[p, s] == fo[p]
