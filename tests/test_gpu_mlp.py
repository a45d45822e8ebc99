"""The learned alpha proposal on the GPU against the FP64 oracle (oracle/mlp.py):
features, FP32 forward and analytic gradient (training arithmetic), Adam,
BF16 tensor-core forward (inference), training, and what the trained
proposal gains over the moment-series start at the same H-error bound."""
import numpy as np
import pytest

import oracle
from oracle import mlp as OM
from paper_1612_05404_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


def _theta(seed=4):
    th = OM.init_params(seed)
    rng = np.random.default_rng(seed)
    th[OM.NH * OM.NIN:OM.NH * OM.NIN + OM.NH] = rng.normal(scale=0.2, size=OM.NH)
    th[-1] = 0.05
    return th


def _cuda(a):
    torch = _torch()
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _X(n, seed=7):
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1, 1, size=(n, OM.NIN))
    X[:, 19] = rng.uniform(-0.2, 1.0, size=n)
    return X


def test_forward_fp32_matches_oracle():
    from paper_1612_05404_gb300 import elbm
    th = _theta().astype(np.float32).astype(np.float64)
    X = _X(1000).astype(np.float32).astype(np.float64)
    o = elbm.mlp_forward(_cuda(X.T), _cuda(th), arith="fp32").cpu().numpy()
    ref, _ = OM.forward(th, X)
    assert np.max(np.abs(o - ref)) <= 1e-5 * (1 + np.max(np.abs(ref)))


def test_forward_bf16_tensor_cores_within_bf16_tolerance():
    """BF16 operands (unit roundoff 2^-8), FP32 accumulation: each layer adds
    a relative error of a few 2^-8 through its operand roundings; over two
    layers the rms error stays below 2^-5 of the rms output and the largest
    below 2^-3 of the largest output."""
    from paper_1612_05404_gb300 import elbm
    th = _theta().astype(np.float32).astype(np.float64)
    X = _X(4133).astype(np.float32).astype(np.float64)  # 129 warp tiles + a ragged tail
    o = elbm.mlp_forward(_cuda(X.T), _cuda(th), arith="bf16_tc").cpu().numpy()
    ref, _ = OM.forward(th, X)
    err = o - ref
    assert np.sqrt(np.mean(err ** 2)) <= 2 ** -5 * np.sqrt(np.mean(ref ** 2))
    assert np.max(np.abs(err)) <= 2 ** -3 * np.max(np.abs(ref))


def test_gradient_matches_oracle_backprop():
    from paper_1612_05404_gb300 import elbm
    th = _theta().astype(np.float32).astype(np.float64)
    X = _X(1000).astype(np.float32).astype(np.float64)  # 7 blocks of 128 + 104
    y = np.random.default_rng(9).normal(size=1000).astype(np.float32).astype(np.float64)
    g, L = elbm.mlp_grad(_cuda(X.T), _cuda(y), _cuda(th))
    g = g.cpu().numpy()
    gref, Lref = OM.grad(th, X, y)
    assert np.linalg.norm(g - gref) <= 1e-4 * np.linalg.norm(gref)
    assert abs(float(L.cpu()[0]) - Lref) <= 1e-5 * Lref


def test_adam_step_matches_oracle():
    from paper_1612_05404_gb300 import elbm
    rng = np.random.default_rng(2)
    th, g = rng.normal(size=OM.NPARAM), rng.normal(size=OM.NPARAM)
    m, v = rng.normal(size=OM.NPARAM) * 0.1, rng.uniform(0, 0.1, size=OM.NPARAM)
    th, g, m, v = (a.astype(np.float32).astype(np.float64) for a in (th, g, m, v))
    tt, tm, tv = _cuda(th), _cuda(m), _cuda(v)
    elbm.mlp_adam(tt, _cuda(g), tm, tv, 7, 1e-3)
    # the kernel's hyper-parameters are FP32 values: give the oracle the same
    f = lambda x: float(np.float32(x))
    rth, rm, rv = OM.adam(th, g, m, v, 7, f(1e-3), f(0.9), f(0.999), f(1e-8))
    # FP32 update: relative error ~1e-6 of the step, plus the rounding of theta
    step = np.abs(rth - th)
    assert np.all(np.abs(tt.cpu().numpy() - rth) <= 1e-5 * step + 2 ** -23 * np.abs(rth) + 1e-9)
    assert np.allclose(tm.cpu().numpy(), rm, rtol=1e-6, atol=1e-8)
    assert np.allclose(tv.cpu().numpy(), rv, rtol=1e-5, atol=1e-9)


def _sites(n_rand=6144):
    cfg, fl = W.drop_in_field(E0=1e-3, n=16, radius=4.5, precision="fp64")
    s = oracle.Sim(cfg, fl)
    s.step(4)
    parts = [s.f.reshape(19, -1)] + [W.random_populations(n_rand, amp, seed=50 + i)
                                     for i, amp in enumerate((0.05, 0.1, 0.2, 0.3))]
    return np.concatenate(parts, axis=1)


def test_features_and_targets_match_oracle():
    from paper_1612_05404_gb300 import elbm
    F = _sites(512)
    d32 = (F - W.D3Q19_WEIGHTS[:, None]).astype(np.float32)
    d = _cuda(d32)
    _, _, st, delta = elbm.alpha_eval(d, aprec="fp32", eq_tol=1e-5, with_delta=True)
    X, S = elbm.alpha_features(d)
    Xh, y, keep = elbm.alpha_harvest(d)
    f32 = (W.D3Q19_WEIGHTS.astype(np.float32)[:, None] + d32).astype(np.float64)
    D = delta.cpu().numpy().astype(np.float64)
    Xr, Sr = OM.features(f32, D)
    assert np.max(np.abs(X.cpu().numpy().T - Xr)) <= 4e-6
    assert np.allclose(S.cpu().numpy(), Sr, rtol=2e-6)
    # harvested features use the kernel's fast division: a few ulps
    assert np.max(np.abs(Xh.cpu().numpy().T - Xr)) <= 4e-6
    k = keep.cpu().numpy().astype(bool)
    assert k.sum() > 1000 and np.all(Sr[k] >= OM.S_MIN * (1 - 1e-6))
    # targets (alpha* - alpha_c)/S^3 against the oracle's FP64 root and start.
    # The FP32 start alpha_c = -2 h'(0)/M2 (1 + ...) inherits the relative
    # rounding of h'(0), about 2^-21 (1 + sum|Delta ln(f/(w rho))| / |h'(0)|)
    # (its terms may cancel), and of the moments; the guarded root is off by
    # |h| / |h'| <= 1e-10 rho / |h'(alpha*)|; both are divided by S^3
    idx = np.flatnonzero(k)[::17]
    h0 = np.array([oracle.h_prime0(3, f32[:, i], D[:, i]) for i in idx])
    rho = f32[:, idx].sum(axis=0)
    tla = np.array([np.sum(np.abs(D[:, i] * np.log(f32[:, i] / (W.D3Q19_WEIGHTS * rho[j]))))
                    for j, i in enumerate(idx)])
    ar = np.array([oracle.alpha(3, f32[:, i], D[:, i], 1e-5)[0] for i in idx])
    hp = np.array([(oracle.h(3, f32[:, i], D[:, i], a * (1 + 1e-7)) - oracle.h(3, f32[:, i], D[:, i], a)) / (a * 1e-7)
                   for i, a in zip(idx, ar)])
    yr = OM.target(f32[:, idx], D[:, idx], h0, ar)
    ac_err = 2.0 ** -21 * 2.0 * (4.0 + tla / np.abs(h0))
    tol = (ac_err + 1.5e-10 * rho / np.abs(hp)) / Sr[idx] ** 3 + 1e-4
    assert np.all(np.abs(y.cpu().numpy()[idx] - np.clip(yr, -8, 8)) <= tol)


def test_trained_proposal_saves_newton_evaluations_at_the_same_h_error():
    """Train on harvested pairs with the project's kernels, then compare on
    held-out sites: the fraction of sites whose FP32 Newton needs more than one
    evaluation of h (status 5) drops with the trained proposal, while every
    root keeps H-error <= 1e-10 rho (float-float guard) in both runs."""
    torch = _torch()
    from paper_1612_05404_gb300 import elbm
    F = _sites(8192)
    rng = np.random.default_rng(0)
    perm = rng.permutation(F.shape[1])
    tr, te = perm[: int(0.8 * len(perm))], perm[int(0.8 * len(perm)):]
    d_all = (F - W.D3Q19_WEIGHTS[:, None]).astype(np.float32)
    X, y, keep = elbm.alpha_harvest(_cuda(d_all[:, tr]))
    k = keep.bool()
    Xk, yk = X[:, k].contiguous(), y[k].contiguous()
    assert Xk.shape[1] > 5000
    theta = _cuda(OM.init_params(3))
    m, v = torch.zeros_like(theta), torch.zeros_like(theta)
    _, L0 = elbm.mlp_grad(Xk, yk, theta)
    hist = elbm.mlp_train(Xk, yk, theta, m, v, 0, 3000, 512, 2e-3, seed=12345)
    _, L1 = elbm.mlp_grad(Xk, yk, theta)
    L0, L1 = float(L0.cpu()[0]), float(L1.cpu()[0])
    assert np.isfinite(hist.cpu().numpy()).all()
    assert L1 < 0.05 * L0, (L0, L1)

    dte = _cuda(d_all[:, te])
    a_n, he_n, st_n, _ = elbm.alpha_eval(dte, aprec="fp32", eq_tol=1e-5)
    a_l, he_l, st_l, _ = elbm.alpha_eval(dte, aprec="fp32", eq_tol=1e-5, mlp=theta)
    st_n, st_l = st_n.cpu().numpy(), st_l.cpu().numpy()
    assert not np.any(st_n == 4) and not np.any(st_l == 4)
    roots = np.isin(st_n, (0, 5))
    assert np.array_equal(roots, np.isin(st_l, (0, 5)))
    assert he_n.cpu().numpy()[roots].max() <= 1e-10 and he_l.cpu().numpy()[roots].max() <= 1e-10
    # the same root within the bound's reach
    da = np.abs(a_n.cpu().numpy() - a_l.cpu().numpy())[roots]
    assert da.max() <= 1e-6
    multi_n = np.mean(st_n[roots] == 5)
    multi_l = np.mean(st_l[roots] == 5)
    assert multi_l < 0.7 * multi_n, (multi_n, multi_l)


def _rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def test_learned_alpha_in_the_step_keeps_parity_and_h_error():
    """alpha_mode "learned" inside the FP32 step: the proposal (trained here on
    pairs harvested from the same GPU simulation) only starts the Newton
    iteration, so the step keeps its FP32 parity with the FP64 oracle, which
    computes the plain root, and every site keeps H-error <= 1e-10 rho."""
    torch = _torch()
    from paper_1612_05404_gb300 import elbm
    cfg, fields = W.drop_in_field(E0=1e-3, n=16, radius=4.5, precision="fp32")
    cfg.update(store_macro=1, alpha_precision="fp32")
    g0 = elbm.Sim(cfg, fields)
    pops = []
    for _ in range(6):
        g0.step(1)
        pops.append(g0.get("f").reshape(19, -1))
    g0.close()
    d = (np.concatenate(pops, axis=1) - W.D3Q19_WEIGHTS[:, None]).astype(np.float32)
    X, y, keep = elbm.alpha_harvest(_cuda(d))
    k = keep.bool()
    Xk, yk = X[:, k].contiguous(), y[k].contiguous()
    assert Xk.shape[1] > 500
    theta = _cuda(OM.init_params(5))
    m, v = torch.zeros_like(theta), torch.zeros_like(theta)
    elbm.mlp_train(Xk, yk, theta, m, v, 0, 1500, 256, 2e-3, seed=777)

    g = elbm.Sim(dict(cfg, alpha_mode="learned", mlp=theta), fields)
    o = oracle.Sim(dict(cfg, poisson_tol=1e-13), fields)
    for t in range(4):
        g.step(1)
        o.step(1)
        e5 = dict(rho=_rel_l2(g.get("rho"), o.rho), phi=_rel_l2(g.get("phi"), o.phi))
        assert max(e5.values()) < 1e-5, (t, e5)
        dg = g.diag()
        assert dg["max_h_error"] <= 1e-10 and dg["n_guard_failed"] == 0, dg
        assert 0 <= dg["n_learned_fallback"] <= 16 ** 3
    g.close()


@pytest.mark.parametrize("autotune", [0, 1])
def test_fused_learned_start_equals_alpha_eval(autotune):
    """The learned proposal runs inside the collision, only in warps with a
    site that starts from it (S >= 2^-5). The alpha it gives must be the
    alpha that elbm_alpha_eval computes with the same network on the same
    populations (the same Delta, proposal and Newton iteration), bit for bit,
    whatever block shape the launch uses (autotune picks among 128x1 ..
    8x16; warps of two-dimensional blocks span several rows); only a root
    the float-float guard took may differ in its last bits (the collision
    sums the guard's pairs over groups of 1 to 8 lanes, elbm_alpha_eval on
    one), and it still solves the exact equation to 1e-10 rho."""
    torch = _torch()
    from paper_1612_05404_gb300 import elbm
    cfg, fields = W.drop_in_field(E0=1e-3, n=24, radius=6.5, precision="fp32")
    cfg.update(store_macro=1, alpha_precision="fp32", autotune=autotune)
    theta = _cuda(OM.init_params(11)) * 0.3
    g = elbm.Sim(dict(cfg, alpha_mode="learned", mlp=theta), fields)
    g.step(4)
    f = g.get("f").reshape(19, -1)
    g.step(1)
    a_step = g.get("alpha")
    dg = g.diag()
    g.close()
    d = _cuda((f - W.D3Q19_WEIGHTS[:, None]).astype(np.float32))
    a, he, st, _ = elbm.alpha_eval(d, aprec="fp32", eq_tol=cfg["alpha_eq_tol"], mlp=theta)
    a = a.cpu().numpy()
    st = st.cpu().numpy()
    _, S = elbm.alpha_features(d)
    hard = S.cpu().numpy() >= 2 ** -5
    assert hard.sum() > 100  # sites that start from the network
    diff = np.flatnonzero(a_step != a)
    assert len(diff) <= dg["n_guarded"], (len(diff), dg["n_guarded"])
    fx = W.D3Q19_WEIGHTS[:, None] + (f - W.D3Q19_WEIGHTS[:, None]).astype(np.float32).astype(np.float64)
    c, _, _ = oracle.lattice(3)
    for i in diff:
        rho = fx[:, i].sum()
        D = oracle.feq(3, rho, (c.T @ fx[:, i]) / rho) - fx[:, i]
        for al in (a_step[i], a[i]):
            assert abs(oracle.h(3, fx[:, i], D, al)) / rho <= 1e-10, (i, al)
    assert dg["max_h_error"] <= 1e-10 and dg["n_guard_failed"] == 0
