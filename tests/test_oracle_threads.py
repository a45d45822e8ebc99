"""The oracle's site-parallel loops: results are the same bit for bit for
any number of threads (every global sum is taken serially in site order)."""
import numpy as np
import pytest

import oracle
from paper_1612_05404_gb300 import workloads as W


def _run(cfg, fields, steps, threads):
    oracle.set_threads(threads)
    sim = oracle.Sim(cfg, fields)
    sim.step(steps)
    out = dict(f=sim.f.copy(), phi=sim.phi.copy(), rho=sim.rho.copy(), u=sim.u.copy(), q=sim.q.copy(),
               alpha=sim.alpha.copy(), nu=sim.nu.copy(), diag=sim.diag.copy())
    if sim.g is not None:
        out["g"] = sim.g.copy()
    return out


@pytest.mark.parametrize("case", ["drop_transport", "jet_xi_full"])
def test_threads_bit_identical(case):
    if case == "drop_transport":
        cfg, fields = W.drop_in_field(E0=1e-3, n=12, radius=3.5, precision="fp64")
        cfg["poisson_tol"] = 1e-10
    else:
        cfg, fields = W.jet(shape=(16, 16, 24), nozzle_r=3, wall=1, nozzle_len=5, precision="fp64")
        cfg.update(force_el="full", poisson_tol=1e-10)
    n0 = oracle.set_threads(0)
    try:
        one = _run(cfg, fields, 3, 1)
        many = _run(cfg, fields, 3, 4)
    finally:
        oracle.set_threads(n0)
    for k in one:
        assert np.array_equal(one[k], many[k]), k
