#!/usr/bin/env python
"""Throughput of the charged entropic lattice Boltzmann step on GB300.

Metric: lattice-site updates per second (MLUPS) of the whole step, and the
HBM roofline fraction of the fused collision kernel.

Workload "drop64" (default): the leaky-dielectric drop between electrodes,
four independent 64^3 D3Q19 lattices, one per applied field
E0 = 1e-4, 4e-4, 7e-4, 1e-3 along z; drop radius 12, liquid / vapour
densities 2.0 / 0.16 (G = -5), Carreau n = 0.6, lambda = 10, transported
free charge (eps ratio 2, sigma ratio 10), populations stored as FP32
deviations with FP32 arithmetic. One bench step = one time step of each of
the four lattices. The 256 MiB L2 flush between timed steps is outside the
timed region; the four lattices together (about 190 MB of state) also exceed
the 129 MB L2.

Runs on N GPUs as N independent replicas (weak scaling): each rank steps
its own four lattices, no data-path collective.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ELBM MLUPS & frac of 8 TB/s HBM; learned-α vs Newton-α at equal H-error"
NOMINAL_HBM_GBS = 8000.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="drop64", choices=["drop64"])
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32", "bf16"])
    ap.add_argument("--alpha-precision", default="fp32", choices=["fp64", "fp32", "fp32_fast"])
    ap.add_argument("--alpha-mode", default="entropic", choices=["entropic", "bgk"],
                    help="bgk: alpha = 2 (the method without its entropic step; for cost attribution)")
    ap.add_argument("--instances", type=int, default=4, help="lattices per step (E0 sweep values)")
    ap.add_argument("--no-graph", action="store_true", help="issue each step from the host (profilers see every launch)")
    ap.add_argument("--launch", default="batch", choices=["batch", "streams"],
                    help="batch: all lattices in one graph per step; streams: one graph per lattice per stream")
    ap.add_argument("--span", type=int, default=0,
                    help="batch: steps per graph launch (ELBM_BATCH_SPAN, 1..16); timed launches cover that "
                         "many steps; 0: the span that covers --steps in the fewest launches")
    ap.add_argument("--pipeline", default="on", choices=["on", "off"],
                    help="batch: odd-position lattices run half a step ahead (ELBM_BATCH_PIPELINE)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-alpha-compare", action="store_true",
                    help="skip the learned-alpha vs Newton-alpha comparison")
    ap.add_argument("--boxes", type=int, default=512,
                    help="batched-droplets comparison: number of boxes (0 skips it)")
    ap.add_argument("--no-jet", action="store_true", help="skip the electrified-jet measurement")
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


def workload_cfgs(args):
    from paper_1612_05404_gb300 import workloads as W
    out = []
    for E0 in W.E0_SWEEP[len(W.E0_SWEEP) - args.instances:]:
        cfg, fields = W.drop_in_field(E0=E0, precision=args.precision)
        cfg.update(alpha_precision=args.alpha_precision, alpha_mode=args.alpha_mode, store_macro=0, diag_every=1,
                   poisson_check_every=8, graph=0 if args.no_graph else 1)
        out.append((cfg, fields))
    return out


def cpu_sample(steps=3):
    """The oracle, as it stands, on a 32^3 lattice of the same physics
    (E0 = 1e-3, drop radius 6): one untimed step (cold potential), then
    `steps` timed steps, single-threaded."""
    import oracle
    from paper_1612_05404_gb300 import workloads as W
    cfg, fields = W.drop_in_field(E0=1e-3, n=32, radius=6.0, precision="fp32")
    sim = oracle.Sim(cfg, fields)
    sim.step(1)
    t0 = time.perf_counter()
    sim.step(steps)
    dt = time.perf_counter() - t0
    return 32 ** 3 * steps / dt / 1e6, dt, f"oracle FP64, 32^3 drop-in-field (E0=1e-3), {steps} steps after 1 untimed"


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


def run_reference(args, rank):
    if rank != 0:
        return None
    import oracle
    from paper_1612_05404_gb300 import workloads as W
    cfg, fields = W.drop_in_field(E0=1e-3, n=32, radius=6.0, precision="fp32")
    sim = oracle.Sim(cfg, fields)
    sim.step(max(args.warmup, 1))
    t0 = time.perf_counter()
    sim.step(args.steps)
    dt = time.perf_counter() - t0
    v = 32 ** 3 * args.steps / dt / 1e6
    return {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "drop-in-field, sample: one 32^3 lattice (E0=1e-3) of the 64^3 x4 bench workload",
                   "oracle": "plain FP64 C, single thread"},
        "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": 1, "kind": "oracle",
                         "sample": f"32^3 lattice, {args.steps} steps after {max(args.warmup, 1)} untimed"},
        "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_ours(args, rank, world, local_rank):
    import ctypes
    import numpy as np
    import torch
    from concurrent.futures import ThreadPoolExecutor
    from paper_1612_05404_gb300 import build, elbm
    torch.cuda.set_device(local_rank)
    build.build()
    cfgs = workload_cfgs(args)
    nx, ny, nz = cfgs[0][0]["shape"]
    N = nx * ny * nz
    if args.launch == "batch":
        # all lattices in one CUDA graph per step (autotuned launch shapes)
        for c, _ in cfgs:
            c.update(autotune=1, profile=0)
        sims = [elbm.Sim(c, f) for c, f in cfgs]
        batch = elbm.Batch(sims, pipeline=args.pipeline == "on", span=span_of(args))
        step_all = lambda m=1: batch.step(m)
        streams = None
    else:
        # one CUDA stream per lattice, stepped from a thread pool (the library
        # call releases the GIL)
        streams = [torch.cuda.Stream() for _ in cfgs]
        sims = [elbm.Sim(c, f, stream=ctypes.c_void_p(st.cuda_stream)) for (c, f), st in zip(cfgs, streams)]
        pool = ThreadPoolExecutor(max_workers=len(sims))
        step_all = lambda m=1: list(pool.map(lambda s: s.step(m), sims))
    # timed launches: `span` steps per graph launch (batch), the rest one step
    # at a time; exactly args.steps steps in all
    span = span_of(args) if args.launch == "batch" else 1
    chunks = [span] * (args.steps // span) + [1] * (args.steps % span)
    for _ in range(args.warmup):
        step_all()
    torch.cuda.synchronize()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    times = []
    sweeps0 = sum(s.diag()["poisson_sweeps_total"] for s in sims)
    with ClockSampler(local_rank) as clk:
        for m in chunks:
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            if streams:
                for st in streams:
                    st.wait_event(e0)
            step_all(m)
            if streams:
                cur = torch.cuda.current_stream()
                for st in streams:
                    cur.wait_event(st.record_event())
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
    sweeps = sum(s.diag()["poisson_sweeps_total"] for s in sims) - sweeps0
    torch.cuda.synchronize()
    total_ms = sum(times)
    if world > 1:
        total_ms = max_over_ranks(total_ms, "cuda")
        dist.barrier()
    diag = [s.diag() for s in sims]
    if args.launch == "batch":
        batch.close()
    else:
        pool.shutdown()
    for s in sims:
        s.close()
    value = job_mlups(len(sims) * N * args.steps, world, total_ms)

    # the collision kernel alone: one lattice (E0 = 1e-3), each pass timed with
    # CUDA events on its stream (three section graphs per step)
    c1, f1 = cfgs[-1]
    c1 = dict(c1, profile=1, autotune=1)
    prof = elbm.Sim(c1, f1)
    prof.step(args.warmup)
    p0 = prof.pass_times()
    prof.step(args.steps)
    p1 = prof.pass_times()
    prof.close()
    d = {k: p1[k] - p0[k] for k in p0}
    bf = {"fp64": 8, "fp32": 4, "bf16": 2}[args.precision]
    bs = 8 if args.precision == "fp64" else 4
    bytes_site = 2 * 19 * bf + 3 * bs + 14 * bs  # f read+write, rho/phi/q reads, g read+write
    coll_ms = d["collide_ms"] / max(d["collide_launches"], 1)
    achieved = N * bytes_site / (coll_ms * 1e-3) / 1e9
    peak, peak_kind = peaks()
    shares = {k: d[k] / max(d["moments_ms"] + d["poisson_ms"] + d["collide_ms"] + d["reduce_ms"], 1e-30)
              for k in ("moments_ms", "poisson_ms", "collide_ms", "reduce_ms")}
    launches_per_step = d["launches"] / max(d["steps"], 1)
    out = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32", "bf16": "bf16"}[args.precision],
        "data": "synthetic",
        "config": {"workload": f"drop-in-field: {len(sims)} x 64^3 D3Q19 lattices (E0 sweep 1e-4..1e-3), "
                               "transported charge, Carreau n=0.6",
                   "sites_per_step": len(sims) * N, "population_storage": {"fp64": "fp64", "fp32": "fp32 deviation from w",
                                          "bf16": "bf16, relative to the site density"}[args.precision],
                   "alpha_arithmetic": args.alpha_precision,
                   "l2": "256 MiB flush between timed launches (outside timing); lattice state %.0f MB > L2 (129 MB)"
                         % (len(sims) * N * (2 * 19 * {"fp64": 8, "fp32": 4, "bf16": 2}[args.precision] + 2 * 7 * 4
                                             + 6 * (8 if args.precision == "fp64" else 4)) / 1e6),
                   "timed_launch_steps": span,
                   "poisson": "multigrid V(2,2), red-black Gauss-Seidel, tol 1e-6 (FP32 floor stop), warm start extrapolated from the two previous potentials",
                   "poisson_vcycles_per_step": sweeps / max(args.steps, 1) / len(sims),
                   "launch": ("CUDA graphs of %d step(s) for all lattices (batch), autotuned block shapes" % span
                              + (", odd lattices half a step ahead" if args.pipeline == "on" else "")
                              if args.launch == "batch" else "one graph per lattice on concurrent streams"),
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "kernel": "k_collide", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_kind,
                     "frac_of_8TBps": achieved / NOMINAL_HBM_GBS,
                     # ncu dram__bytes_read.sum + dram__bytes_write.sum of one 64^3 FP32
                     # launch of this kernel (cold caches)
                     "traffic": 32.51e6 if args.precision == "fp32" else None,
                     "bytes_per_site": bytes_site, "avg_launch_ms": coll_ms,
                     "timed": "one 64^3 lattice alone, CUDA events around each collision launch"},
        "pass_share": shares,
        # kernels of the timed launches: per lattice and step those of the
        # one-step graph, less the diagnostics finalize that a graph of m
        # steps runs once instead of m times
        "gpu_launches": int(round(len(sims) * sum(m * launches_per_step - (m - 1) for m in chunks))),
        "alpha": {"max_h_error_device": max(x["max_h_error"] for x in diag), "h_error_bound": 1e-10,
                  "guarded_sites_last_step": sum(x["n_guarded"] for x in diag),
                  "guard_failed_last_step": sum(x["n_guard_failed"] for x in diag),
                  "noroot": sum(x["n_noroot"] for x in diag), "clipped": sum(x["n_clipped"] for x in diag)},
        "clocks": clk.summary(),
    }
    return out, cfgs, N


def e2e_run(args, cfgs, N):
    """The same metric end to end through the public API with host buffers,
    on the headline's launch path: elbm_init of every lattice from host
    arrays (H2D), the batch, warm-up and timed steps with every step's
    diagnostics (the step's result) copied to pinned host memory, the final
    density fields read back, elbm_free."""
    import numpy as np
    import torch
    from paper_1612_05404_gb300 import elbm
    h2d = 0
    for c, f in cfgs:
        c.update(profile=0, autotune=1)
        h2d += sum(v.nbytes for v in f.values() if hasattr(v, "nbytes"))
    n_steps = args.warmup + args.steps
    diag = [torch.empty(elbm.NDIAG, dtype=torch.float64).pin_memory() for _ in cfgs]
    diag_np = [d.numpy() for d in diag]
    rho = [np.empty(N) for _ in cfgs]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sims = [elbm.Sim(c, f) for c, f in cfgs]
    batch = elbm.Batch(sims, pipeline=args.pipeline == "on")
    t_init = time.perf_counter() - t0
    for _ in range(n_steps):
        batch.step(1)
        for s, d in zip(sims, diag_np):
            s.fields(elbm.F_DIAG, d)
    for s, r in zip(sims, rho):
        s.fields(elbm.F_RHO, r)
    batch.close()
    for s in sims:
        s.close()
    dt = time.perf_counter() - t0
    d2h = len(cfgs) * (elbm.NDIAG * 8 + N * 8 / n_steps)
    return {"value": len(cfgs) * N * n_steps / dt / 1e6, "unit": "MLUPS",
            "h2d_bytes_per_step": int(h2d / n_steps), "d2h_bytes_per_step": int(d2h),
            "init_seconds": t_init,
            "timed": "init from host arrays + batch + %d steps with per-step diagnostics read to pinned "
                     "host memory + final density read + free" % n_steps}


def _timed_steps(sims, streams, pool, steps, warmup):
    """Device time (ms) of `steps` steps of all lattices, after `warmup`."""
    import torch
    for _ in range(warmup):
        list(pool.map(lambda s: s.step(1), sims))
    torch.cuda.synchronize()
    p0 = [s.pass_times() for s in sims]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    total = 0.0
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for st in streams:
            st.wait_event(e0)
        list(pool.map(lambda s: s.step(1), sims))
        cur = torch.cuda.current_stream()
        for st in streams:
            cur.wait_event(st.record_event())
        e1.record()
        torch.cuda.synchronize()
        total += e0.elapsed_time(e1)
    p1 = [s.pass_times() for s in sims]
    d = {k: sum(b[k] - a[k] for a, b in zip(p0, p1)) for k in p0[0]}
    return total, d


def alpha_compare(args, N):
    """Learned-alpha vs Newton-alpha on the bench workload at one H-error
    bound (<= 1e-10 rho): the FP64 Newton root, the FP32 Newton root with the
    float-float guard, and the FP32 iteration started from the learned
    proposal (trained here on the GPU: pairs harvested from the first steps of
    the E0 = 1e-3 lattice, the project's training kernels); step throughput,
    collision time per launch, device H-error and fallbacks."""
    import ctypes
    from concurrent.futures import ThreadPoolExecutor
    import numpy as np
    import torch
    from paper_1612_05404_gb300 import elbm
    from paper_1612_05404_gb300 import workloads as W
    out = {}
    # training pairs from the plain run of one lattice
    t0 = time.perf_counter()
    cfg, fields = W.drop_in_field(E0=1e-3, precision=args.precision)
    cfg.update(alpha_precision="fp32", store_macro=0, diag_every=1, poisson_check_every=8, graph=1)
    sim = elbm.Sim(cfg, fields)
    Xs, ys = [], []
    for k in range(24):
        sim.step(1)
        if k % 3 == 2:
            d = torch.from_numpy((sim.get("f").reshape(19, -1) - W.D3Q19_WEIGHTS[:, None]).astype(np.float32)).cuda()
            X, y, keep = elbm.alpha_harvest(d)
            kk = keep.bool()
            Xs.append(X[:, kk])
            ys.append(y[kk])
    sim.close()
    X = torch.cat(Xs, dim=1).contiguous()
    y = torch.cat(ys).contiguous()
    rng = np.random.default_rng(20161209)
    import math
    lim1, lim2, lim3 = math.sqrt(6 / 84), math.sqrt(6 / 128), math.sqrt(6 / 65)
    theta = torch.zeros(elbm.MLP_NPARAM, dtype=torch.float32)
    theta[:1280] = torch.from_numpy(rng.uniform(-lim1, lim1, 1280).astype(np.float32))
    theta[1344:5440] = torch.from_numpy(rng.uniform(-lim2, lim2, 4096).astype(np.float32))
    theta[5504:5568] = torch.from_numpy(rng.uniform(-lim3, lim3, 64).astype(np.float32))
    theta = theta.cuda()
    m, v = torch.zeros_like(theta), torch.zeros_like(theta)
    hist = elbm.mlp_train(X, y, theta, m, v, 0, 4000, 1024, 2e-3, seed=20161209)
    torch.cuda.synchronize()
    h = hist.cpu().numpy()
    out["training"] = {"pairs": int(X.shape[1]), "steps": 4000, "batch": 1024,
                       "loss_first": float(h[:50].mean()), "loss_last": float(h[-50:].mean()),
                       "seconds": time.perf_counter() - t0,
                       "data": "pairs harvested every 3rd of the first 24 steps of the E0=1e-3 lattice, S >= 2^-5"}

    def run(mode, aprec, steps):
        cfgs = workload_cfgs(args)
        streams = [torch.cuda.Stream() for _ in cfgs]
        sims = []
        for (c, f), st in zip(cfgs, streams):
            c.update(profile=1, alpha_mode=mode, alpha_precision=aprec)
            if mode == "learned":
                c["mlp"] = theta
            sims.append(elbm.Sim(c, f, stream=ctypes.c_void_p(st.cuda_stream)))
        pool = ThreadPoolExecutor(max_workers=len(sims))
        ms, d = _timed_steps(sims, streams, pool, steps, args.warmup)
        diag = [s.diag() for s in sims]
        for s in sims:
            s.close()
        pool.shutdown()
        return {"mlups": len(sims) * N * steps / (ms * 1e-3) / 1e6, "ms_per_step": ms / steps,
                "collide_ms_per_launch": d["collide_ms"] / max(d["collide_launches"], 1),
                "max_h_error_device": max(x["max_h_error"] for x in diag),
                "guarded_sites_last_step": sum(x["n_guarded"] for x in diag),
                "learned_fallback_sites_last_step": sum(x["n_learned_fallback"] for x in diag),
                "steps": steps}

    out["newton_fp64"] = run("entropic", "fp64", max(2, args.steps // 5))
    out["newton_fp32_guarded"] = run("entropic", "fp32", args.steps)
    out["learned_fp32_guarded"] = run("learned", "fp32", args.steps)
    out["h_error_bound"] = 1e-10
    out["speedup_learned_vs_newton_fp32"] = out["learned_fp32_guarded"]["mlups"] / out["newton_fp32_guarded"]["mlups"]
    out["speedup_learned_vs_newton_fp64"] = out["learned_fp32_guarded"]["mlups"] / out["newton_fp64"]["mlups"]
    return out


def jet_run(args):
    """The electrified jet at full size: 128 x 128 x 512, nozzle of radius 8
    injecting Carreau liquid (n = 0.5, lambda = 20) at 0.02 along z, E0 = 5e-4,
    xi-form charge, BF16 deviation storage with FP32 arithmetic, guarded FP32
    alpha, multigrid Poisson with the nozzle as a conductor."""
    import torch
    from paper_1612_05404_gb300 import elbm
    from paper_1612_05404_gb300 import workloads as W
    cfg, fields = W.jet(precision="bf16")
    cfg.update(alpha_precision="fp32", poisson_solver="mg", graph=1, diag_every=1, autotune=1)
    N = cfg["shape"][0] * cfg["shape"][1] * cfg["shape"][2]
    sim = elbm.Sim(cfg, fields)
    del fields
    sim.step(args.warmup)
    torch.cuda.synchronize()
    total, cycles, herr, guarded = 0.0, 0.0, 0.0, 0.0
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        sim.step(1)
        e1.record()
        torch.cuda.synchronize()
        total += e0.elapsed_time(e1)
        d = sim.diag()
        cycles += d["poisson_sweeps"]
        herr = max(herr, d["max_h_error"])
        guarded += d["n_guarded"]
    sim.close()
    return {"workload": "electrified jet 128x128x512, nozzle r=8, Carreau n=0.5 lambda=20, E0=5e-4, xi-form charge",
            "storage": "bf16, relative to the site density", "sites": N, "mlups": N * args.steps / (total * 1e-3) / 1e6,
            "ms_per_step": total / args.steps, "poisson": "multigrid, nozzle as conductor",
            "poisson_vcycles_per_step": cycles / args.steps, "max_h_error_device": herr,
            "guarded_site_fraction": guarded / (N * args.steps)}


def batched_compare(args):
    """Batched droplets (uneven boxes, one CUDA graph launch per step for all)
    against the same boxes stepped one at a time, at the same H-error bound
    (guarded FP32 alpha), FP32 storage, autotuned launch shapes."""
    import torch
    from paper_1612_05404_gb300 import elbm
    from paper_1612_05404_gb300 import workloads as W
    params = W.batched_droplet_params(n_boxes=args.boxes)
    t0 = time.perf_counter()
    sims = []
    for edge, E0, nc in params:
        cfg, fields = W.batched_droplet(edge, E0, nc, precision="fp32")
        cfg.update(alpha_precision="fp32", autotune=1, graph=1, diag_every=1)
        sims.append(elbm.Sim(cfg, fields))
    t_init = time.perf_counter() - t0
    sites = sum(e ** 3 for e, _, _ in params)
    t0 = time.perf_counter()
    batch = elbm.Batch(sims, pipeline=args.pipeline == "on", span=span_of(args))
    t_capture = time.perf_counter() - t0
    batch.step(args.warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    batch.step(args.steps)
    e1.record()
    torch.cuda.synchronize()
    ms_b = e0.elapsed_time(e1) / args.steps
    hmax_b = max(s.diag()["max_h_error"] for s in sims)
    batch.close()
    # the same boxes one at a time: each box's own step graph, launched and
    # finished before the next box starts
    single_ms = 0.0
    for s in sims:
        s.step(1)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        s.step(2)
        b.record()
        torch.cuda.synchronize()
        single_ms += a.elapsed_time(b) / 2
    hmax_s = max(s.diag()["max_h_error"] for s in sims)
    for s in sims:
        s.close()
    return {"boxes": len(params), "sites": sites, "edges": sorted(set(e for e, _, _ in params)),
            "batched": {"mlups": sites / (ms_b * 1e-3) / 1e6, "ms_per_step": ms_b, "max_h_error_device": hmax_b,
                        "graph_launches_per_step": 1.0 / span_of(args), "pipelined": args.pipeline == "on"},
            "one_at_a_time": {"mlups": sites / (single_ms * 1e-3) / 1e6, "ms_per_step": single_ms,
                              "max_h_error_device": hmax_s},
            "speedup_batched_vs_single": single_ms / ms_b,
            "init_seconds": t_init, "capture_seconds": t_capture,
            "workload": "batched droplets: periodic cubic boxes, edge over {24..96} step 8 except 72, 88, "
                        "R = edge/4, E0 ~ U[0,1e-3] along z, Carreau n ~ U[0.5,1], lambda 10, transported charge"}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        res = run_reference(args, rank)
        if res is not None:
            print(json.dumps(res), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    res, cfgs, N = run_ours(args, rank, world, local_rank)
    if not args.no_e2e:
        res["e2e"] = e2e_run(args, cfgs, N)
        res["e2e"]["value"] *= world
    if rank == 0 and world == 1 and not args.no_alpha_compare and args.precision != "fp64":
        res["alpha_compare"] = alpha_compare(args, N)
    if rank == 0 and world == 1 and args.boxes > 0:
        res["batched_compare"] = batched_compare(args)
    if rank == 0 and world == 1 and not args.no_jet:
        res["jet"] = jet_run(args)
    if rank == 0 and world == 1 and not args.no_cpu:
        v, dt, sample = cpu_sample()
        res["cpu_baseline"] = {"value": v, "unit": "MLUPS", "cores": 1, "kind": "oracle", "sample": sample}
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
