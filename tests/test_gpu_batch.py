"""Batched lattices (elbm_batch_create): one CUDA graph launch per step for
instances of uneven size and parameters must reproduce the same instances run
one by one, bit for bit (same kernels, launch shapes and reduction order);
the autotuned launch shape changes only the grouping of the block sums."""
import numpy as np
import pytest

import oracle
from paper_1612_05404_gb300 import workloads as W

pytestmark = pytest.mark.gpu

BOXES = [(16, 2e-4, 0.6), (24, 9e-4, 1.0), (32, 5e-4, 0.8)]


def _make(precision="fp32", **extra):
    from paper_1612_05404_gb300 import elbm
    sims = []
    for edge, E0, nc in BOXES:
        cfg, fields = W.batched_droplet(edge, E0, nc, precision=precision)
        cfg.update(extra)
        sims.append(elbm.Sim(cfg, fields))
    return sims


def test_batch_reproduces_single_instances_bitwise():
    from paper_1612_05404_gb300 import elbm
    single = _make()
    for s in single:
        s.step(5)
    grouped = _make()
    batch = elbm.Batch(grouped)
    assert batch.step(2) >= 0
    assert batch.step(3) >= 0
    for a, b in zip(single, grouped):
        for name in ("rho", "phi", "q", "f"):
            assert np.array_equal(a.get(name), b.get(name)), name
        assert a.diag()["step"] == b.diag()["step"] == 5
    batch.close()


def test_batched_fp64_instance_matches_oracle():
    from paper_1612_05404_gb300 import elbm
    sims = _make(precision="fp64")
    batch = elbm.Batch(sims)
    batch.step(3)
    edge, E0, nc = BOXES[1]
    cfg, fields = W.batched_droplet(edge, E0, nc, precision="fp64")
    o = oracle.Sim(cfg, fields)
    o.step(3)
    g = sims[1]
    for name, ref in (("rho", o.rho), ("phi", o.phi), ("q", o.q)):
        v = g.get(name)
        assert np.linalg.norm(v - ref) <= 1e-10 * np.linalg.norm(ref), name
    batch.close()


def test_autotuned_shapes_keep_the_results():
    from paper_1612_05404_gb300 import elbm
    plain = _make(precision="fp64")
    tuned = _make(precision="fp64", autotune=1)
    for s in plain:
        s.step(3)
    batch = elbm.Batch(tuned)
    batch.step(3)
    for a, b in zip(plain, tuned):
        for name in ("rho", "phi"):
            x, y = a.get(name), b.get(name)
            assert np.linalg.norm(x - y) <= 1e-11 * np.linalg.norm(x), name
    batch.close()


def test_stepping_an_instance_alone_is_refused():
    from paper_1612_05404_gb300 import elbm
    sims = _make()
    batch = elbm.Batch(sims)
    batch.step(1)
    sims[0].step(1)
    with pytest.raises(elbm.ElbmError):
        batch.step(1)
    batch.close()


def test_pipelined_batch_keeps_populations_bitwise():
    """ELBM_BATCH_PIPELINE: every instance stores the populations of the
    one-at-a-time run; an instance at an odd position has already solved the
    next step's moments and potential, so its density, charge and potential
    are those of the single run one step later."""
    from paper_1612_05404_gb300 import elbm
    s5, s6 = _make(), _make()
    for s in s5:
        s.step(5)
    for s in s6:
        s.step(6)
    grouped = _make()
    batch = elbm.Batch(grouped, pipeline=True)
    assert batch.step(2) >= 0
    assert batch.step(3) >= 0
    for i, (a5, a6, b) in enumerate(zip(s5, s6, grouped)):
        assert np.array_equal(a5.get("f"), b.get("f")), i
        moments = a6 if i % 2 else a5
        for name in ("rho", "phi", "q"):
            assert np.array_equal(moments.get(name), b.get(name)), (i, name)
        assert b.diag()["step"] == 5
    batch.close()
    # stepped alone after the batch, the instance ahead repeats its solve
    grouped[1].step(1)
    assert np.linalg.norm(grouped[1].get("f") - s6[1].get("f")) <= 1e-5 * np.linalg.norm(s6[1].get("f"))


def test_batch_reports_each_instance_status():
    """The step's status words come back through the batch graph: a
    non-finite instance makes the batch step fail with ELBM_E_NUMERIC, and a
    Poisson solve stopped at its cap gives the warning, as for a lone
    instance."""
    from paper_1612_05404_gb300 import elbm
    cfg = W.base_params(shape=(8, 8, 8), precision="fp64", charge_model="transport", poisson_maxit=50)
    rho = np.ones(512)
    rho[100] = -1.0
    good = _make()
    bad = elbm.Sim(cfg, dict(rho=rho))
    batch = elbm.Batch(good + [bad])
    with pytest.raises(elbm.ElbmError) as ei:
        batch.step(1)
    assert ei.value.code == elbm.E_NUMERIC
    batch.close()

    cfg2, fields2 = W.charged_drop_at_rest(n=12, radius=3.5)
    cfg2.update(precision="fp64", poisson_solver="sor", poisson_maxit=3, poisson_check_every=1)
    capped = elbm.Sim(cfg2, fields2)
    batch = elbm.Batch(_make() + [capped])
    assert batch.step(1) == elbm.W_POISSON_NOCONV
    assert capped.diag()["poisson_sweeps"] == 3
    batch.close()


@pytest.mark.parametrize("pipeline", [False, True])
def test_span_graphs_reproduce_one_step_launches_bitwise(pipeline):
    """ELBM_BATCH_SPAN(4): graphs of four consecutive steps run the same
    kernels in the same order per instance as four one-step launches; a
    step count that is not a multiple of the span ends with one-step
    launches."""
    from paper_1612_05404_gb300 import elbm
    one, spanned = _make(), _make()
    b1 = elbm.Batch(one, pipeline=pipeline)
    b4 = elbm.Batch(spanned, pipeline=pipeline, span=4)
    assert b1.step(7) >= 0
    assert b4.step(7) >= 0
    for a, b in zip(one, spanned):
        for name in ("rho", "phi", "q", "f"):
            assert np.array_equal(a.get(name), b.get(name)), name
        assert a.diag() == b.diag()
    b1.close()
    b4.close()


def _uniform_kick(**extra):
    """A periodic 16^3 lattice in one uniform state far from equilibrium
    (f_p = w_p (1 + e_p), e_p ~ U(-0.1, 0.1), the same at every site; no
    Shan-Chen coupling): the first collision takes the entropic root at every
    site (S = 0.14), after it the lattice sits within S < 1e-3 of equilibrium,
    below the near-equilibrium shortcut of 0.05, so every later step takes
    alpha = 2 without a root (the oracle: 4096 shortcuts from the second
    step on)."""
    from paper_1612_05404_gb300 import elbm
    cfg = W.base_params(shape=(16, 16, 16), G=0.0, Gw=0.0, precision="fp32", alpha_precision="fp32",
                        alpha_eq_tol=0.05)
    cfg.update(extra)
    _, w = elbm.velocity_set()
    e = np.random.default_rng(5).uniform(-0.1, 0.1, 19)
    fs = w * (1.0 + e)
    N = 16 ** 3
    fields = dict(rho=np.full(N, fs.sum()), f=np.repeat(fs[:, None], N, axis=1).reshape(-1))
    return elbm.Sim(cfg, fields)


def test_span_graph_reports_the_guard_failures_of_its_first_step():
    """A graph of four steps forms the full diagnostics on its last step
    only; the sticky record of the steps before it must carry their guard
    failures and H-error into those diagnostics. With an H-error target of
    1e-30 (below what the float-float guard resolves) every root of the
    first step ends as a guard failure; steps 2-4 take no root."""
    from paper_1612_05404_gb300 import elbm
    one = _uniform_kick(alpha_h_tol=1e-30)
    b1 = elbm.Batch([one], span=1)
    assert b1.step(1) >= 0
    d1 = one.diag()
    assert d1["n_guard_failed"] == 16 ** 3 and d1["n_shortcut"] == 0
    assert d1["flags_undiagnosed"] == 0
    assert b1.step(1) >= 0
    d2 = one.diag()
    assert d2["n_guard_failed"] == 0 and d2["n_shortcut"] == 16 ** 3 and d2["max_h_error"] == 0.0
    b1.close()

    four = _uniform_kick(alpha_h_tol=1e-30)
    b4 = elbm.Batch([four], span=4)
    assert b4.step(4) >= 0
    d = four.diag()
    assert d["step"] == 4 and d["n_shortcut"] == 16 ** 3
    assert d["flags_undiagnosed"] == 2.0          # bit 1: a guard failure on an earlier step
    assert d["n_guard_failed"] == 1.0             # none on the last step, plus the flag
    assert d["max_h_error"] == d1["max_h_error"]  # the first step's, carried over
    # the record restarts with the diagnostics that folded it in
    assert b4.step(4) >= 0
    d = four.diag()
    assert d["flags_undiagnosed"] == 0.0 and d["n_guard_failed"] == 0.0 and d["max_h_error"] == 0.0
    b4.close()


def test_span_graph_max_h_error_covers_every_step():
    """At the default target (1e-10) the H-error maximum that a four-step
    graph reports equals the maximum of the four steps' own diagnostics in
    one-step launches, bit for bit (here the first step's: the others take
    no root); the host-issued path with diagnostics every fourth step
    reports the same."""
    from paper_1612_05404_gb300 import elbm
    one = _uniform_kick()
    b1 = elbm.Batch([one], span=1)
    herr = []
    for _ in range(4):
        assert b1.step(1) >= 0
        herr.append(one.diag()["max_h_error"])
    b1.close()
    assert herr[0] > 0.0 and herr[0] <= 1e-10 and max(herr[1:]) == 0.0
    four = _uniform_kick()
    b4 = elbm.Batch([four], span=4)
    assert b4.step(4) >= 0
    assert four.diag()["max_h_error"] == max(herr) and four.diag()["flags_undiagnosed"] == 0.0
    b4.close()
    host = _uniform_kick(graph=0, diag_every=4)
    assert host.step(4) == elbm.OK
    assert host.diag()["max_h_error"] == max(herr)
