"""Writes tests/golden/paper_drop_field_2d.json from the oracle alone: the
paper's charged drop in a uniform field (Sec. III A) with its protocol, on
its 320^2 D2Q9 lattice in FP64: 1000 steps at rest (the first experiment),
then E_ext = 0.5 along x from that equilibrium, read every 250 steps up to
t = 1250. Stored per reading: the maximum mean curvature K on the interface
contour (rho at the middle of the extreme densities, within a tenth of their
span), the largest and smallest charge alteration delta_q = q - q_{K=0}
(Eq. surface-q2 with the curvature term off, renormalised), the liquid's
centroid along x and its aspect ratio, and the density at sampled sites.
About 80 minutes on 8 host cores:
    python tests/golden/make_paper_drop_field_2d.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1612_05404_gb300 import workloads as W  # noqa: E402

N_SIDE = 320
REST_STEPS = 1000
READ_EVERY = 250
FIELD_STEPS = 1250
E_EXT = 0.5
# sampled sites: the row through the drop's centre along the field, and a column across it
SAMPLE_SITES = [x + N_SIDE * 160 for x in range(100, 300, 5)] + [220 + N_SIDE * y for y in range(100, 221, 5)]


def measures(cfg, mask, rho):
    q, K, _ = oracle.charge_field(cfg, mask, rho)
    q0, _, _ = oracle.charge_field(dict(cfg, K_d=1e300), mask, rho)
    dq = q - q0
    r = rho.reshape(N_SIDE, N_SIDE)
    rl, rv = float(r.max()), float(r.min())
    contour = np.abs(rho - 0.5 * (rl + rv)) < 0.1 * (rl - rv)
    w = np.clip(r - rv, 0.0, None)
    y, x = np.mgrid[0:N_SIDE, 0:N_SIDE]
    m = w.sum()
    cx, cy = (w * x).sum() / m, (w * y).sum() / m
    aspect = np.sqrt((w * (x - cx) ** 2).sum() / (w * (y - cy) ** 2).sum())
    return dict(K_max_contour=float(K[contour].max()), dq_plus=float(dq.max()), dq_minus=float(dq.min()),
                centroid_x=float(cx), aspect=float(aspect), rho_min=rv, rho_max=rl,
                rho_samples=[float(rho[s]) for s in SAMPLE_SITES])


def main():
    cfg, fl = W.paper_drop_2d()
    cfg.update(poisson_tol=1e-10, poisson_check_every=8, store_macro=1)
    rest = oracle.Sim(cfg, fl)
    rest.step(REST_STEPS)
    field_cfg = dict(cfg, E_ext=(E_EXT, 0.0, 0.0))
    sim = oracle.Sim(field_cfg, dict(fl, f=rest.f.copy()))
    out = dict(about="oracle (FP64) run of the paper's drop in a field, Sec. III A; written by "
                     "tests/golden/make_paper_drop_field_2d.py",
               rest_steps=REST_STEPS, E_ext=E_EXT, poisson_tol=cfg["poisson_tol"], sample_sites=SAMPLE_SITES,
               readings={"0": measures(cfg, fl["mask"], rest.rho)})
    for t in range(READ_EVERY, FIELD_STEPS + 1, READ_EVERY):
        sim.step(READ_EVERY)
        out["readings"][str(t)] = measures(cfg, fl["mask"], sim.rho)
        print(t, {k: v for k, v in out["readings"][str(t)].items() if k != "rho_samples"}, flush=True)
    with open(os.path.join(ROOT, "tests", "golden", "paper_drop_field_2d.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
