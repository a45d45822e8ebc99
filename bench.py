#!/usr/bin/env python
"""Throughput of the charged entropic lattice Boltzmann step on GB300.

Metric: lattice-site updates per second (MLUPS) of the whole step, the HBM
roofline fraction of its dominant kernel, and the learned alpha proposal
against the Newton root at the same H-error bound.

Workload "jet4" (default): the electrified jet at 256 x 256 x 768 D3Q19
sites (50.3 M): a nozzle of radius 8 injects Carreau liquid (n = 0.5,
lambda = 20) at 0.02 along z into vapour, E0 = 5e-4 along z, xi-form free
charge, multigrid potential with the nozzle as a conductor; populations
stored in BF16 relative to the site density with FP32 arithmetic; entropic
alpha by the learned proposal (a 20-64-64-1 network trained here, on the
GPU, on (f, alpha) pairs harvested from the drop-in-field and 128 x 128 x
512 jet runs) followed by the FP32 Newton iteration and the float-float
guard, certified to |h(alpha)|/rho <= 1e-10 against the exact equation.
Every timed step computes its diagnostics (mass, momentum, charge, alpha
statistics, H-error maximum, non-finite count) and checks its status. The
lattice state (8.4 GB) exceeds the 129 MB L2, so no flush is needed.

Runs on N GPUs as N independent replicas (weak scaling): each rank steps its
own lattice, no data-path collective; rank 0 also runs the secondary
measurements when N = 1.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ELBM MLUPS & frac of 8 TB/s HBM; learned-α vs Newton-α at equal H-error"
NOMINAL_HBM_GBS = 8000.0
JET4_SHAPE = (256, 256, 768)
JET3_SHAPE = (128, 128, 512)
SAMPLE_SHAPE = (48, 48, 128)  # the oracle's sample of the jet physics (multi-core baseline)
SAMPLE1_SHAPE = (32, 32, 96)  # the same, single thread; also the reference arm's sample


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--alpha-mode", default="learned", choices=["learned", "entropic"],
                    help="headline alpha: learned proposal + guarded Newton, or guarded Newton alone")
    ap.add_argument("--train-steps", type=int, default=4000, help="Adam steps of the proposal's training")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=100,
                    help="steps of the end-to-end run (elbm_init from host arrays inside the timed region)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the secondary measurements (alpha comparison, drop, batch, jet 128)")
    ap.add_argument("--boxes", type=int, default=512, help="batched-droplets comparison: boxes (0 skips it)")
    ap.add_argument("--batched-steps", type=int, default=40, help="batched-droplets comparison: timed steps")
    ap.add_argument("--ncu-case", default="", choices=["", "jet128", "jet4"],
                    help="profiling run for ncu: the 128x128x512 (or 256x256x768) jet with learned alpha, "
                         "steps issued from the host (every kernel a separate launch), fixed block shape; "
                         "--warmup + --steps steps, no timing")
    ap.add_argument("--span", type=int, default=0,
                    help="drop-in-field batch: steps per graph launch besides span 1 (0: the span that "
                         "covers --steps in the fewest launches)")
    return ap.parse_args()


def span_of(args):
    """Steps per batch graph launch: --span, or the span up to 16 that covers
    the timed steps in the fewest launches (full spans plus single steps),
    with the smallest remainder among those (10 for 20 steps)."""
    if args.span > 0:
        return args.span
    n = max(args.steps, 1)
    return min(range(1, 17), key=lambda s: (n // s + n % s, n % s, s))


def max_over_ranks(ms, device):
    """The slowest rank's time of the timed region (every rank the same
    number of units): all-reduce MAX over the default process group (NCCL on
    the GPUs; any backend whose tensors live on `device`)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(units_per_rank, world, ms_max):
    """Whole-job throughput: every rank's replicas (weak scaling, no data-path
    collective) over the slowest rank's time."""
    return units_per_rank * world / (ms_max * 1e-3) / 1e6


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def host_cpu():
    model = platform.processor() or platform.machine()
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                k = line.split(":")[0].strip().lower()
                if k in ("model name", "cpu model", "hardware"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    try:
        lscpu = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in lscpu.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"model": model, "nproc": os.cpu_count(), "machine": platform.machine()}


class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not self.path:
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
_FIELDS = {}


def jet_case(shape, alpha_mode="learned", aprec="fp32", theta=None, **extra):
    """Config dict and (cached) initial fields of the jet at `shape`: BF16
    storage relative to the site density, FP32 arithmetic, multigrid with
    the nozzle as a conductor, graphs with per-step diagnostics."""
    from paper_1612_05404_gb300 import workloads as W
    key = tuple(shape)
    if key not in _FIELDS:
        _FIELDS[key] = W.jet(shape=shape, precision="bf16")
    cfg, fields = _FIELDS[key]
    cfg = dict(cfg, alpha_precision=aprec, alpha_mode=alpha_mode, poisson_solver="mg", graph=1, diag_every=1,
               autotune=1, store_macro=0, profile=0)
    if alpha_mode == "learned":
        cfg["mlp"] = theta
    cfg.update(extra)
    return cfg, fields


def sites(shape):
    return shape[0] * shape[1] * shape[2]


def timed_steps(sim, steps, clocks=None):
    """Device time (ms) of `steps` steps of one lattice, one CUDA-event pair
    around them (each elbm_step waits for its step and checks its status)."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        sim.step(1)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


# ---------------------------------------------------------------------------
# the learned proposal: pairs harvested from configs 2 and 3, trained on the GPU
# ---------------------------------------------------------------------------
def _harvest(sim, keep_mask=None):
    """Training pairs of every fluid site of a lattice (FP32 deviations of its
    populations through elbm_fields, elbm_alpha_harvest on the GPU)."""
    import numpy as np
    import torch
    from paper_1612_05404_gb300 import elbm
    from paper_1612_05404_gb300 import workloads as W
    f = sim.get("f").reshape(19, -1)
    fluid = f.sum(0) > 0
    d = torch.from_numpy(np.ascontiguousarray(f[:, fluid] - W.D3Q19_WEIGHTS[:, None]).astype(np.float32)).cuda()
    del f
    X, y, keep = elbm.alpha_harvest(d)
    kk = keep.bool()
    return X[:, kk].contiguous(), y[kk].contiguous(), int(fluid.sum())


def train_proposal(args):
    """(theta, report): the proposal's network trained with the project's
    kernels (elbm_mlp_train, minibatch Adam) on pairs harvested from the
    drop-in-field (config 2: 64^3, E0 = 1e-3 and 7e-4, FP32) and the jet
    (config 3: 128 x 128 x 512, BF16) during their first steps; sites with
    S = max|Delta/f| >= 2^-5, where the proposal is used."""
    import math
    import numpy as np
    import torch
    from paper_1612_05404_gb300 import elbm
    from paper_1612_05404_gb300 import workloads as W
    t0 = time.perf_counter()
    Xs, ys, seen, src = [], [], 0, {}
    for E0 in (1e-3, 7e-4):
        cfg, fields = W.drop_in_field(E0=E0, precision="fp32")
        cfg.update(alpha_precision="fp32", store_macro=0, diag_every=1, poisson_check_every=8, graph=1)
        sim = elbm.Sim(cfg, fields)
        for k in range(30):
            sim.step(1)
            if k % 3 == 2:
                X, y, n = _harvest(sim)
                Xs.append(X); ys.append(y); seen += n
                src["drop64"] = src.get("drop64", 0) + int(y.numel())
        sim.close()
    cfg, fields = jet_case(JET3_SHAPE, alpha_mode="entropic")
    sim = elbm.Sim(cfg, fields)
    for k in range(30):
        sim.step(1)
        if k % 10 == 9:
            X, y, n = _harvest(sim)
            Xs.append(X); ys.append(y); seen += n
            src["jet128"] = src.get("jet128", 0) + int(y.numel())
    sim.close()
    X = torch.cat(Xs, dim=1).contiguous()
    y = torch.cat(ys).contiguous()
    del Xs, ys
    t_h = time.perf_counter() - t0
    rng = np.random.default_rng(20161209)
    lim1, lim2, lim3 = math.sqrt(6 / 84), math.sqrt(6 / 128), math.sqrt(6 / 65)
    theta = torch.zeros(elbm.MLP_NPARAM, dtype=torch.float32)
    theta[:1280] = torch.from_numpy(rng.uniform(-lim1, lim1, 1280).astype(np.float32))
    theta[1344:5440] = torch.from_numpy(rng.uniform(-lim2, lim2, 4096).astype(np.float32))
    theta[5504:5568] = torch.from_numpy(rng.uniform(-lim3, lim3, 64).astype(np.float32))
    theta = theta.cuda()
    m, v = torch.zeros_like(theta), torch.zeros_like(theta)
    hist = elbm.mlp_train(X, y, theta, m, v, 0, args.train_steps, 1024, 2e-3, seed=20161209)
    torch.cuda.synchronize()
    h = hist.cpu().numpy()
    return theta, {"pairs": int(X.shape[1]), "pairs_by_source": src, "sites_harvested": seen,
                   "adam_steps": args.train_steps, "batch": 1024, "lr": 2e-3,
                   "loss_first": float(h[:50].mean()), "loss_last": float(h[-50:].mean()),
                   "harvest_seconds": t_h, "seconds": time.perf_counter() - t0,
                   "data": "every 3rd of the first 30 steps of two 64^3 drops in field (E0 = 1e-3, 7e-4) and "
                           "steps 10, 20, 30 of the 128x128x512 jet; fluid sites with S >= 2^-5 (the others "
                           "use the moment-series start, not the network)"}


# ---------------------------------------------------------------------------
# the headline: config 4
# ---------------------------------------------------------------------------
# DRAM bytes (read + write) per site of one collision launch, measured by ncu
# (dram__bytes_read.sum + dram__bytes_write.sum) on the 128x128x512 jet with
# the learned proposal: 814.066688 MB over 8,388,608 sites. Valid for the
# collision kernel as it stood for that capture.
COLLIDE_DRAM_BYTES_PER_SITE = 814.066688e6 / 8388608


def bytes_per_site_collide():
    """Algorithmic bytes of one collision launch per site, BF16 storage:
    populations read and written (2 x 19 x 2), the reference-density plane
    read and written (2 x 4), the psi, phi and q planes read (3 x 4), the
    node-kind mask (1). (The learned proposal runs inside this kernel.)"""
    return 2 * 19 * 2 + 2 * 4 + 3 * 4 + 1


def run_headline(args, rank, world, local_rank, theta):
    import torch
    N = sites(JET4_SHAPE)
    from paper_1612_05404_gb300 import elbm
    cfg, fields = jet_case(JET4_SHAPE, alpha_mode=args.alpha_mode, theta=theta)
    sim = elbm.Sim(cfg, fields)
    for _ in range(args.warmup):
        sim.step(1)
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    d0 = sim.diag()
    with ClockSampler(local_rank) as clk:
        ms = timed_steps(sim, args.steps)
    d1 = sim.diag()
    sim.close()
    total_ms = ms
    if world > 1:
        total_ms = max_over_ranks(ms, "cuda")
        import torch.distributed as dist
        dist.barrier()
    value = job_mlups(N * args.steps, world, total_ms)
    diag = {"max_h_error_device_last_step": d1["max_h_error"], "guard_failed_last_step": d1["n_guard_failed"],
            "guarded_sites_last_step": d1["n_guarded"], "learned_fallback_sites_last_step": d1["n_learned_fallback"],
            "nonfinite": d1["n_nonfinite"], "noroot_last_step": d1["n_noroot"],
            "poisson_vcycles_per_step": (d1["poisson_sweeps_total"] - d0["poisson_sweeps_total"]) / args.steps,
            "mass_drift_rel": abs(d1["mass"] - d0["mass"]) / d0["mass"]}
    return value, total_ms, clk.summary(), diag


def roofline(args, theta):
    """The collision kernel of the headline alone: the same lattice issued
    step by step with CUDA events around each pass (profile mode); its
    average launch time against its algorithmic bytes."""
    from paper_1612_05404_gb300 import elbm
    N = sites(JET4_SHAPE)
    cfg, fields = jet_case(JET4_SHAPE, alpha_mode=args.alpha_mode, theta=theta, graph=0, profile=1)
    sim = elbm.Sim(cfg, fields)
    sim.step(max(args.warmup, 3))
    p0 = sim.pass_times()
    n = max(5, min(args.steps, 10))
    sim.step(n)
    p1 = sim.pass_times()
    sim.close()
    d = {k: p1[k] - p0[k] for k in p0}
    launches = d["collide_launches"]
    coll_ms = d["collide_ms"] / max(launches, 1)  # the collision kernel (+ the tiny diagnostics finalize)
    bs = bytes_per_site_collide()
    achieved = N * bs / (coll_ms * 1e-3) / 1e9
    peak, kind = peaks()
    tot = d["moments_ms"] + d["poisson_ms"] + d["collide_ms"] + d["reduce_ms"]
    out = {"bound": "hbm", "kernel": "k_collide", "achieved": achieved, "peak": peak, "unit": "GB/s",
           "frac": achieved / peak, "peak_source": kind, "frac_of_8TBps": achieved / NOMINAL_HBM_GBS,
           # ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch of this kernel on the
           # 128x128x512 jet, scaled by sites to this lattice (the traffic is per site)
           "traffic": COLLIDE_DRAM_BYTES_PER_SITE * N,
           "traffic_source": "ncu, one k_collide launch on the 128x128x512 jet (462.44 + 351.63 MB over "
                             "8,388,608 sites), scaled by the site count",
           "bytes_per_site": bs, "avg_launch_ms": coll_ms,
           "timed": "256x256x768 jet, steps issued one by one, CUDA events around each pass (profile mode)"}
    shares = {"moments_charge": d["moments_ms"] / tot, "poisson": d["poisson_ms"] / tot,
              "collide": d["collide_ms"] / tot}
    launches_per_step = d["launches"] / max(d["steps"], 1)
    return out, shares, launches_per_step, {k: d[k] / max(d["steps"], 1) for k in
                                            ("moments_ms", "poisson_ms", "collide_ms")}


def e2e_run(args, theta):
    """The same metric end to end through the public API with host buffers:
    elbm_init from host arrays (fields and the network's parameters
    uploaded), --e2e-steps steps with every step's diagnostics copied to
    pinned host memory and read, the final density read back, elbm_free, all
    inside the timed region (the one-time initialisation is amortised over
    the run's steps, as in a simulation of the jet)."""
    import numpy as np
    import torch
    from paper_1612_05404_gb300 import elbm
    N = sites(JET4_SHAPE)
    cfg, fields = jet_case(JET4_SHAPE, alpha_mode=args.alpha_mode, theta=theta)
    theta_host = theta.cpu() if theta is not None else None
    h2d = sum(v.nbytes for v in fields.values() if hasattr(v, "nbytes"))
    h2d += theta_host.numel() * 4 if theta_host is not None else 0
    n_steps = args.e2e_steps
    diag = torch.empty(elbm.NDIAG, dtype=torch.float64).pin_memory()
    diag_np = diag.numpy()
    rho = np.empty(N)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if theta_host is not None:
        cfg = dict(cfg, mlp=theta_host.cuda(non_blocking=False))
    sim = elbm.Sim(cfg, fields)
    t_init = time.perf_counter() - t0
    for _ in range(n_steps):
        sim.step(1)
        sim.fields(elbm.F_DIAG, diag_np)
    sim.fields(elbm.F_RHO, rho)
    sim.close()
    dt = time.perf_counter() - t0
    d2h = elbm.NDIAG * 8 + N * 8 / n_steps
    return {"value": N * n_steps / dt / 1e6, "unit": "MLUPS", "h2d_bytes_per_step": int(h2d / n_steps),
            "d2h_bytes_per_step": int(d2h), "init_seconds": t_init, "steps": n_steps,
            "timed": "elbm_init from host arrays (fields + network) + %d steps, each with its diagnostics read "
                     "from pinned host memory + final density read + elbm_free" % n_steps}


# ---------------------------------------------------------------------------
# secondary measurements (rank 0, N = 1)
# ---------------------------------------------------------------------------
def alpha_compare(args, theta, learned_ms):
    """Learned proposal vs the Newton root on the headline workload at one
    bound (|h|/rho <= 1e-10 against the exact equation): guarded FP32 Newton
    alone, and the FP64 Newton root (two steps; 1/64-rate FP64 on this part)."""
    from paper_1612_05404_gb300 import elbm
    N = sites(JET4_SHAPE)
    out = {}
    for name, mode, aprec, steps in (("newton_fp32_guarded", "entropic", "fp32", args.steps),
                                     ("newton_fp64", "entropic", "fp64", 2)):
        cfg, fields = jet_case(JET4_SHAPE, alpha_mode=mode, aprec=aprec)
        sim = elbm.Sim(cfg, fields)
        sim.step(args.warmup if aprec == "fp32" else 1)
        ms = timed_steps(sim, steps)
        d = sim.diag()
        sim.close()
        out[name] = {"mlups": N * steps / (ms * 1e-3) / 1e6, "ms_per_step": ms / steps, "steps": steps,
                     "max_h_error_device_last_step": d["max_h_error"], "guarded_sites_last_step": d["n_guarded"]}
    out["learned_fp32_guarded"] = {"mlups": N * args.steps / (learned_ms * 1e-3) / 1e6,
                                   "ms_per_step": learned_ms / args.steps, "steps": args.steps}
    out["speedup_learned_vs_newton_fp32"] = (out["learned_fp32_guarded"]["mlups"]
                                             / out["newton_fp32_guarded"]["mlups"])
    out["speedup_learned_vs_newton_fp64"] = out["learned_fp32_guarded"]["mlups"] / out["newton_fp64"]["mlups"]
    out["h_error_bound"] = "1e-10 rho, exact equation of the stored populations"
    return out


def alpha_stage(theta):
    """Where the proposal is used: the alpha root alone (elbm_alpha_eval) on
    held-out strongly non-equilibrium sites (S >= 2^-5) of a drop in field not
    seen in training (E0 = 4e-4, step 33): guarded FP32 Newton from the
    moment-series start vs from the learned proposal, same bound."""
    import numpy as np
    import torch
    from paper_1612_05404_gb300 import elbm
    from paper_1612_05404_gb300 import workloads as W
    cfg, fields = W.drop_in_field(E0=4e-4, precision="fp32")
    cfg.update(alpha_precision="fp32", store_macro=0, diag_every=1, poisson_check_every=8, graph=1)
    sim = elbm.Sim(cfg, fields)
    sim.step(33)
    f = sim.get("f").reshape(19, -1)
    sim.close()
    d = torch.from_numpy(np.ascontiguousarray(f - W.D3Q19_WEIGHTS[:, None]).astype(np.float32)).cuda()
    _, S = elbm.alpha_features(d)
    hard = torch.nonzero(S >= 2 ** -5).flatten()
    dh = d[:, hard].contiguous()
    reps = max(1, int(2_000_000 // max(dh.shape[1], 1)))
    dh = dh.repeat(1, reps).contiguous()  # enough sites to time the kernel
    res = {}
    for name, mlp in (("newton", None), ("learned", theta)):
        for _ in range(2):
            a, he, st, _ = elbm.alpha_eval(dh, aprec="fp32", eq_tol=1e-5, mlp=mlp)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(5):
            a, he, st, _ = elbm.alpha_eval(dh, aprec="fp32", eq_tol=1e-5, mlp=mlp)
        e1.record()
        torch.cuda.synchronize()
        stn = st.cpu().numpy()
        root = np.isin(stn, (0, 5))
        res[name] = {"ns_per_site": e0.elapsed_time(e1) / 5 * 1e6 / dh.shape[1],
                     "multi_evaluation_fraction": float(np.mean(stn[root] == 5)),
                     "max_h_error_reported": float(he.cpu().numpy()[root].max()),
                     "guard_failed": int(np.sum(stn == 4))}
    res["hard_sites"] = int(hard.numel())
    res["timed_sites"] = int(dh.shape[1])
    res["speedup_learned_vs_newton"] = res["newton"]["ns_per_site"] / res["learned"]["ns_per_site"]
    return res


def fp64_configs(args):
    """Configs 1 and 2 in FP64 (storage, arithmetic and the alpha root, FP64
    Newton): the charged drop at rest (32^3 periodic, transported charge,
    Newtonian) and one 64^3 drop in field (E0 = 1e-3, Carreau n = 0.6), each
    alone, one CUDA graph per step, diagnostics every step."""
    import torch
    from paper_1612_05404_gb300 import elbm
    from paper_1612_05404_gb300 import workloads as W
    out = {}
    cases = (("config1_drop_at_rest_32", W.charged_drop_at_rest(precision="fp64")),
             ("config2_drop_in_field_64", W.drop_in_field(E0=1e-3, precision="fp64")))
    for name, (cfg, fields) in cases:
        cfg = dict(cfg, alpha_precision="fp64", graph=1, diag_every=1, autotune=1)
        sim = elbm.Sim(cfg, fields)
        sim.step(args.warmup)
        ms = timed_steps(sim, args.steps)
        d = sim.diag()
        n = sites(cfg["shape"])
        sim.close()
        out[name] = {"mlups": n * args.steps / (ms * 1e-3) / 1e6, "ms_per_step": ms / args.steps, "sites": n,
                     "max_h_error_device": d["max_h_error"], "poisson_resid": d["poisson_resid"]}
    out["workload"] = "FP64 storage, arithmetic and alpha (Newton), multigrid to 1e-13"
    return out


def poisson64(args):
    """The Poisson chain of one lone 64^3 drop in field (E0 = 1e-3, FP32,
    multigrid, warm), as the step runs it: CUDA events around each pass
    (section graphs), V-cycles per step, device time per V-cycle (the
    warm-start extrapolation and the stop tests included) and kernel
    launches per step."""
    from paper_1612_05404_gb300 import elbm
    from paper_1612_05404_gb300 import workloads as W
    cfg, fields = W.drop_in_field(E0=1e-3, precision="fp32")
    cfg.update(alpha_precision="fp32", store_macro=0, diag_every=1, poisson_check_every=8, graph=1, autotune=1,
               profile=1)
    sim = elbm.Sim(cfg, fields)
    sim.step(args.warmup)
    p0 = sim.pass_times()
    sim.step(args.steps)
    p1 = sim.pass_times()
    sim.close()
    d = {k: p1[k] - p0[k] for k in p0}
    n = max(d["steps"], 1)
    cyc = d["sweeps"] / n
    return {"poisson_ms_per_step": d["poisson_ms"] / n, "vcycles_per_step": cyc,
            "ms_per_vcycle": d["poisson_ms"] / n / max(cyc, 1e-30), "launches_per_step": d["launches"] / n,
            "step_ms": (d["moments_ms"] + d["poisson_ms"] + d["collide_ms"] + d["reduce_ms"]) / n,
            "workload": "one 64^3 drop in field, E0 = 1e-3, FP32, multigrid V(2,2), tail of <= 4096 cells in one CTA"}


def drop64(args):
    """Config 2 at full size: four 64^3 drops in field (the E0 sweep), FP32
    storage, guarded FP32 alpha, one batch; graphs of one step (diagnostics
    every step) and of `span` steps (diagnostics on the last)."""
    import torch
    from paper_1612_05404_gb300 import elbm
    from paper_1612_05404_gb300 import workloads as W
    N = 64 ** 3
    out = {}
    for span in sorted({1, span_of(args)}):
        sims = []
        for E0 in W.E0_SWEEP:
            cfg, fields = W.drop_in_field(E0=E0, precision="fp32")
            cfg.update(alpha_precision="fp32", store_macro=0, diag_every=1, poisson_check_every=8, graph=1,
                       autotune=1)
            sims.append(elbm.Sim(cfg, fields))
        batch = elbm.Batch(sims, pipeline=True, span=span)
        batch.step(args.warmup)
        chunks = [span] * (args.steps // span) + [1] * (args.steps % span)
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
        total = 0.0
        for m in chunks:
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            batch.step(m)
            e1.record()
            torch.cuda.synchronize()
            total += e0.elapsed_time(e1)
        batch.close()
        herr = max(s.diag()["max_h_error"] for s in sims)
        for s in sims:
            s.close()
        out[f"span{span}"] = {"mlups": 4 * N * args.steps / (total * 1e-3) / 1e6, "ms_per_step": total / args.steps,
                              "max_h_error_device": herr,
                              "diagnostics": "every step" if span == 1 else f"last of every {span} steps"}
    out["workload"] = "4 x 64^3 drop in field (E0 sweep), FP32, guarded FP32 alpha, batch, half-step shift"
    return out


def jet128(args):
    """Config 3 at full size: one 128 x 128 x 512 jet, BF16, guarded FP32 Newton."""
    from paper_1612_05404_gb300 import elbm
    N = sites(JET3_SHAPE)
    cfg, fields = jet_case(JET3_SHAPE, alpha_mode="entropic")
    sim = elbm.Sim(cfg, fields)
    sim.step(args.warmup)
    ms = timed_steps(sim, args.steps)
    d = sim.diag()
    sim.close()
    return {"mlups": N * args.steps / (ms * 1e-3) / 1e6, "ms_per_step": ms / args.steps,
            "max_h_error_device_last_step": d["max_h_error"], "guarded_fraction_last_step": d["n_guarded"] / N,
            "workload": "128x128x512 jet, BF16 relative to the site density, guarded FP32 Newton alpha"}


def batched_compare(args, theta):
    """Config 5: batched droplets (boxes of every integer edge in [24, 96],
    learned alpha when a network is given), all boxes one CUDA graph launch
    per step (diagnostics every step) and graphs of 10 steps (diagnostics on
    the last, the sticky record of H-error and failures on every step),
    against the same boxes stepped one at a time with plain guarded Newton
    alpha (and, to isolate the batching, with the same alpha as the batch).
    FP32 storage; the H-error maximum covers every timed step."""
    import torch
    from paper_1612_05404_gb300 import elbm
    from paper_1612_05404_gb300 import workloads as W
    params = W.batched_droplet_params(n_boxes=args.boxes)
    nsites = sum(e ** 3 for e, _, _ in params)
    steps = args.batched_steps

    def make(learned):
        out = []
        for edge, E0, nc in params:
            cfg, fields = W.batched_droplet(edge, E0, nc, precision="fp32")
            cfg.update(alpha_precision="fp32", autotune=1, graph=1, diag_every=1)
            if learned:
                cfg.update(alpha_mode="learned", mlp=theta)
            out.append(elbm.Sim(cfg, fields))
        return out

    def timed_batch(sims, span):
        t0 = time.perf_counter()
        batch = elbm.Batch(sims, pipeline=True, span=span)
        t_cap = time.perf_counter() - t0
        assert batch.step(args.warmup) >= 0
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st = batch.step(steps)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        ds = [s.diag() for s in sims]
        batch.close()
        return {"mlups": nsites / (ms * 1e-3) / 1e6, "ms_per_step": ms, "steps": steps, "status": st,
                "max_h_error_device": max(d["max_h_error"] for d in ds),
                "guard_failed": sum(d["n_guard_failed"] for d in ds),
                "learned_fallback_sites_last_step": sum(d["n_learned_fallback"] for d in ds),
                "graph_launches_per_step": 1.0 / span if steps % span == 0 else None,
                "diagnostics": "every step" if span == 1 else f"last of every {span} steps, sticky record on every step",
                "capture_seconds": t_cap}

    def one_at_a_time(sims, k=5):
        total = 0.0
        for s in sims:
            s.step(1)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            s.step(k)
            b.record()
            torch.cuda.synchronize()
            total += a.elapsed_time(b) / k
        return {"mlups": nsites / (total * 1e-3) / 1e6, "ms_per_step": total, "steps_per_box": k,
                "max_h_error_device": max(s.diag()["max_h_error"] for s in sims),
                "diagnostics": "every step"}

    learned = theta is not None
    t0 = time.perf_counter()
    sims = make(learned)
    t_init = time.perf_counter() - t0
    res = {"boxes": len(params), "sites": nsites, "edges": sorted(set(e for e, _, _ in params)),
           "odd_edge_boxes": sum(1 for e, _, _ in params if e & 1),
           "alpha": "learned proposal + guarded FP32 Newton" if learned else "guarded FP32 Newton",
           "init_seconds": t_init}
    res["batched_span1"] = timed_batch(sims, 1)
    res["batched_span10"] = timed_batch(sims, 10)
    res["one_at_a_time_same_alpha"] = one_at_a_time(sims)
    for s in sims:
        s.close()
    if learned:
        sims = make(False)
        res["one_at_a_time_newton"] = one_at_a_time(sims)
        for s in sims:
            s.close()
    else:
        res["one_at_a_time_newton"] = res["one_at_a_time_same_alpha"]
    base = res["one_at_a_time_newton"]["ms_per_step"]
    res["speedup_batched_vs_single_newton"] = base / res["batched_span1"]["ms_per_step"]
    res["speedup_batched_span10_vs_single_newton"] = base / res["batched_span10"]["ms_per_step"]
    res["speedup_batched_vs_single_same_alpha"] = (res["one_at_a_time_same_alpha"]["ms_per_step"]
                                                   / res["batched_span1"]["ms_per_step"])
    res["workload"] = ("batched droplets: periodic cubic boxes, edge uniform over the integers 24..96, R = edge/4, "
                       "E0 ~ U[0,1e-3] along z, Carreau n ~ U[0.5,1], lambda 10, transported charge, FP32")
    return res


# ---------------------------------------------------------------------------
# the oracle on the host cores
# ---------------------------------------------------------------------------
def oracle_sample(shape, threads, steps, warm=1):
    """The FP64 CPU oracle, as it stands, on a jet of the headline's physics
    at `shape` (nozzle radius 8): `warm` untimed steps, then `steps` timed."""
    import oracle
    from paper_1612_05404_gb300 import workloads as W
    used = oracle.set_threads(threads)
    cfg, fields = W.jet(shape=shape, precision="bf16")
    sim = oracle.Sim(cfg, fields)
    sim.step(warm)
    t0 = time.perf_counter()
    sim.step(steps)
    dt = time.perf_counter() - t0
    return sites(shape) * steps / dt / 1e6, dt, used


def cpu_baseline():
    cores = os.cpu_count() or 1
    v, dt, used = oracle_sample(SAMPLE_SHAPE, cores, 2)
    v1, dt1, _ = oracle_sample(SAMPLE1_SHAPE, 1, 1)
    return {"value": v, "unit": "MLUPS", "cores": used, "kind": "oracle",
            "sample": "FP64 oracle, jet of the headline's physics at %dx%dx%d (nozzle r = 8), 1 untimed + 2 timed "
                      "steps, %d threads (site-parallel loops); MLUPS is per site and step, so it stands for the "
                      "256x256x768 lattice (extrapolated)" % (*SAMPLE_SHAPE, used),
            "seconds": dt, "host": host_cpu(),
            "single_thread": {"value": v1, "unit": "MLUPS", "cores": 1, "seconds": dt1,
                              "sample": "the same physics at %dx%dx%d, 1 untimed + 1 timed step" % SAMPLE1_SHAPE}}


def run_reference(args, rank):
    if rank != 0:
        return None
    import oracle
    from paper_1612_05404_gb300 import workloads as W
    cores = os.cpu_count() or 1
    used = oracle.set_threads(cores)
    cfg, fields = W.jet(shape=SAMPLE1_SHAPE, precision="bf16")
    sim = oracle.Sim(cfg, fields)
    sim.step(max(args.warmup, 1))
    t0 = time.perf_counter()
    sim.step(args.steps)
    dt = time.perf_counter() - t0
    v = sites(SAMPLE1_SHAPE) * args.steps / dt / 1e6
    sample = ("FP64 oracle on a %dx%dx%d jet of the headline's physics (nozzle r = 8), %d steps after %d untimed, "
              "%d threads" % (*SAMPLE1_SHAPE, args.steps, max(args.warmup, 1), used))
    return {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "electrified jet, sample %dx%dx%d of the 256x256x768 headline lattice" % SAMPLE1_SHAPE,
                   "oracle": "plain FP64 C, site-parallel loops"},
        "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": used, "kind": "oracle", "sample": sample,
                         "host": host_cpu()},
        "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def ncu_case(args):
    """The kernels of the headline step as separate launches for ncu: the jet
    at 128x128x512 (or the headline's 256x256x768), BF16 storage, learned
    alpha with a seeded Glorot-initialised network scaled by 0.01 (the
    kernels' cost does not depend on the weights' values; the proposal only
    starts the certified Newton iteration), multigrid, graph = 0 (the
    Poisson loop from the host: a graph with a conditional node hides its
    kernels from ncu), fixed block shape (no autotuner launches)."""
    import math
    import numpy as np
    import torch
    from paper_1612_05404_gb300 import build, elbm
    build.build()
    torch.cuda.set_device(0)
    rng = np.random.default_rng(1)
    theta = torch.zeros(elbm.MLP_NPARAM, dtype=torch.float32)
    theta[:1280] = torch.from_numpy(rng.uniform(-math.sqrt(6 / 84), math.sqrt(6 / 84), 1280).astype(np.float32))
    theta[1344:5440] = torch.from_numpy(rng.uniform(-math.sqrt(6 / 128), math.sqrt(6 / 128), 4096).astype(np.float32))
    theta[5504:5568] = torch.from_numpy(rng.uniform(-math.sqrt(6 / 65), math.sqrt(6 / 65), 64).astype(np.float32))
    theta = theta.cuda() * 0.01
    shape = (128, 128, 512) if args.ncu_case == "jet128" else JET4_SHAPE
    cfg, fields = jet_case(shape, alpha_mode="learned", theta=theta, graph=0, autotune=0)
    sim = elbm.Sim(cfg, fields)
    sim.step(args.warmup + args.steps)
    torch.cuda.synchronize()
    d = sim.diag()
    sim.close()
    print(json.dumps({"ncu_case": args.ncu_case, "steps": args.warmup + args.steps,
                      "max_h_error": d["max_h_error"], "guarded": d["n_guarded"],
                      "poisson_vcycles_total": d["poisson_sweeps_total"]}), flush=True)


def main():
    args = parse()
    if args.ncu_case:
        ncu_case(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        res = run_reference(args, rank)
        if res is not None:
            print(json.dumps(res), flush=True)
        return
    import torch
    torch.cuda.set_device(local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1612_05404_gb300 import build
    build.build()
    theta, training = (None, None)
    if args.alpha_mode == "learned":
        theta, training = train_proposal(args)
    value, total_ms, clocks, hdiag = run_headline(args, rank, world, local_rank, theta)
    res = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": "electrified jet 256x256x768 D3Q19 (50.3M sites), nozzle r=8, Carreau n=0.5 "
                               "lambda=20, E0=5e-4, xi-form charge",
                   "sites_per_step": sites(JET4_SHAPE),
                   "population_storage": "bf16, relative to the site density", "arithmetic": "fp32",
                   "alpha": ("learned proposal + guarded FP32 Newton" if theta is not None
                             else "guarded FP32 Newton") + ", |h|/rho <= 1e-10 against the exact equation",
                   "diagnostics": "every timed step",
                   "l2": "no flush: lattice state 8.4 GB > L2 (129 MB)",
                   "poisson": "multigrid V(2,2), red-black Gauss-Seidel, tol 1e-6 (FP32 floor stop), nozzle "
                              "as a conductor, warm start extrapolated",
                   "launch": "one CUDA graph per step, the Poisson loop a device-side while node, autotuned "
                             "block shape",
                   "parallelism": f"replicas x{world}"},
        "headline_diagnostics": hdiag,
        "clocks": clocks,
    }
    if training is not None:
        res["training"] = training
    roof, shares, lps, pass_ms = roofline(args, theta)
    res["roofline"] = roof
    res["pass_share"] = shares
    res["pass_ms_per_step"] = pass_ms
    res["gpu_launches"] = int(round(lps * args.steps))
    if not args.no_e2e:
        res["e2e"] = e2e_run(args, theta)
        res["e2e"]["value"] *= world
    if rank == 0 and world == 1 and not args.no_extras:
        if theta is not None:
            res["alpha_compare"] = alpha_compare(args, theta, total_ms)
            res["alpha_stage"] = alpha_stage(theta)
        res["jet128"] = jet128(args)
        res["drop64"] = drop64(args)
        res["poisson64"] = poisson64(args)
        res["fp64_configs"] = fp64_configs(args)
        if args.boxes > 0:
            res["batched_compare"] = batched_compare(args, theta)
    if rank == 0 and world == 1 and not args.no_cpu:
        res["cpu_baseline"] = cpu_baseline()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
