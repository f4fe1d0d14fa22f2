#!/usr/bin/env python3
"""Benchmark of the filtered time-domain Krylov eigensolver on GB300.

One step = one full eigensolve on the workload (every part of the hot path):
weights (eq. weightf), kmax-1 filter applications of L fused leapfrog steps
(eq. 2stepmethod, eq. disc_filtercoeff), M-orthonormalisation (Algorithm 2.5),
Rayleigh-Ritz (eq. projevp) and residual acceptance (eq. res). The default
workload is the 128^3 Kuhn cube (2,048,383 dofs, 30,340,171 entries), interval
[40, 45], L = 600, Krylov dimension 60, FP64.

Metric: GDOF*steps/s = dofs * leapfrog steps / time / 1e9 (whole job, all
ranks). The line also carries the roofline of the fused step kernel, the
oracle timed on the host cores (cpu_baseline) and the end-to-end number
through the C ABI with host buffers (e2e).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl kes|reference]
Under torchrun (N > 1) every rank solves its own replica (its own start
vector); value = all ranks' dof-steps / max-over-ranks time ("weak" scaling).
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "GDOF*steps/s"
FALLBACK_HBM_GBS = 6800.0
STEP_KERNEL_SRC = os.path.join(ROOT, "paper_2402_08515_gb300", "csrc", "kernels_step.cu")
BLOCK_KERNEL_SRC = os.path.join(ROOT, "paper_2402_08515_gb300", "csrc", "kernels_block.cu")


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="cube128_fp64")
    ap.add_argument("--impl", default="kes", choices=["kes", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mode", default="solve", choices=["solve", "filter", "tts", "weights"],
                    help="filter: one filter application only (small profiling runs); tts: time to "
                         "converged eigenpairs at residual 1e-8, FP64 form against the FP32 forms with FP64 "
                         "refinement")
    ap.add_argument("--tts-forms", default="", help="comma-separated subset of the --mode tts forms")
    ap.add_argument("--tts-workloads", default="cube128_fp64,box2m_fp64", help="workloads of --mode tts")
    ap.add_argument("--L", type=int, default=0, help="override the workload's time steps (--mode filter)")
    ap.add_argument("--blk-variant", type=int, default=None,
                    help="fixed block step-kernel launch shape instead of the autotuner's choice")
    ap.add_argument("--variant", type=int, default=None,
                    help="fixed step-kernel launch shape instead of the autotuner's choice")
    return ap.parse_args(argv)


# ----------------------------------------------------------------------------- ranks

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def init_dist(world, backend):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist if world > 1 else None


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, value: float, device=None) -> float:
    """Max of a float over all ranks (timing only; no data-path collective)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, value: float, device=None) -> float:
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return None
        rows = list(csv.reader(open(self.path)))
        os.unlink(self.path)
        sm, smax, names = [], [], set()
        keys = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for k, v in zip(keys, r[5:9]):
                if v.strip().lower() == "active":
                    names.add(k)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(names),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- peaks & profiles

def load_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash(src: str = STEP_KERNEL_SRC) -> str:
    return hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]


def profiled_traffic(workload: str, src: str = STEP_KERNEL_SRC):
    """DRAM bytes per step-kernel launch from the committed ncu summary, if it was taken
    on the current source of that kernel, the file src (else None)."""
    path = os.path.join(ROOT, "profiles", f"step_kernel_{workload}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    h = re.search(r"kernel_source_sha256:\s*([0-9a-f]+)", text)
    t = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not h or not t or h.group(1) != kernel_source_hash(src):
        return None
    return float(t.group(1))


# ----------------------------------------------------------------------------- CPU baseline

def oracle_sample(problem, tau, wl, seconds: float, interval=None):
    """Times the oracle's filter application (as it stands) on a bounded number of
    leapfrog steps of the same workload; returns (GDOF*steps/s, steps, seconds)."""
    import numpy as np
    import oracle as O
    from fe_inputs import start_vectors
    wmin, wmax = interval or (wl.omega_min, wl.omega_max)
    S = problem.to_scipy()
    r = start_vectors(problem.n, 1, wl.seed)[0]
    probe = 3
    t0 = time.perf_counter()
    O.filter_apply(S, problem.m, r, tau, O.alpha_table(wmin, wmax, tau, probe))
    per_step = (time.perf_counter() - t0) / probe
    steps = int(max(3, min(wl.L, seconds / max(per_step, 1e-6))))
    alpha = O.alpha_table(wmin, wmax, tau, steps)
    t0 = time.perf_counter()
    out = O.filter_apply(S, problem.m, r, tau, alpha)
    dt = time.perf_counter() - t0
    assert np.isfinite(out).all()
    return problem.n * steps / dt / 1e9, steps, dt


def cpu_cores_used() -> int:
    # scipy's CSR matvec and numpy's elementwise ops run on one thread
    return 1


def workload_problems(wl):
    built = wl.build()
    return (built if isinstance(built, list) else [built]), isinstance(built, list)


def start_block(problems, b, seed):
    """(b, n_total) start vectors: each mesh draws its own seeded block."""
    import numpy as np
    from fe_inputs import start_vectors
    return np.ascontiguousarray(np.concatenate(
        [start_vectors(p.n, b, seed + 97 * j) for j, p in enumerate(problems)], axis=1))


# ----------------------------------------------------------------------------- kes arm

def run_kes(args):
    import numpy as np
    import torch

    import paper_2402_08515_gb300 as K
    from fe_inputs import WORKLOADS
    from fe_inputs import spectra

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = init_dist(world, "nccl")
    dev = torch.device("cuda", local)
    wl = WORKLOADS[args.workload]
    problems, batch = workload_problems(wl)
    n = sum(p.n for p in problems)
    nnz = sum(p.nnz for p in problems)
    b = wl.b
    stream = torch.cuda.Stream(device=dev)
    ctx = K.Context(problems if batch else problems[0], precision=wl.precision, stream=stream,
                    step_variant=args.variant, blk_variant=args.blk_variant, block_b=b)
    h = ctx.handle
    v0 = start_block(problems, 1, wl.seed)[0]
    omega_pow, gersh = K.kes_estimate_omega_max_batch(h, wl.power_iters, v0)
    taus = wl.cfl * 2.0 / omega_pow
    ivs = [wl.mesh_intervals(p) for p in problems]
    F = len(ivs[0])
    wmin_all = np.array([[a for a, _ in iv] for iv in ivs])
    wmax_all = np.array([[c for _, c in iv] for iv in ivs])
    # the solve searches every interval of a mesh at once when the block splits evenly
    # over them (interval f owns b / F columns); otherwise the first interval only
    F_solve = F if F > 1 and b % F == 0 else 1
    wmin1, wmax1 = wmin_all[:, :F_solve], wmax_all[:, :F_solve]
    K.kes_set_filters_batch(h, wmin1, wmax1, taus, wl.L)
    so = K.kes_solve_opts_default()
    so.kmax, so.tol, so.check_every = wl.kmax, wl.acceptance(), wl.check_every
    R0_host = start_block(problems, b, wl.seed + 1 + 1000 * rank)
    R0_dev = torch.from_numpy(R0_host).to(dev)
    torch.cuda.synchronize()
    if args.mode == "filter":
        L = args.L or wl.L
        K.kes_set_filters_batch(h, wmin1[:, :1], wmax1[:, :1], taus, L)
        out = torch.zeros((1, b, n), dtype=torch.float64, device=dev)
        K.kes_filter_apply(h, R0_dev, out, b)
        K.kes_sync(h)
        st = K.kes_get_stats(h)
        if rank == 0:
            print(json.dumps({"mode": "filter", "workload": args.workload, "L": L, "dofs": n, "b": b,
                              "filter_ms": st["filter_ms"], "step_variant": st["step_variant"],
                              "finite": bool(torch.isfinite(out).all())}))
        ctx.close()
        return

    def solve():
        if b == 1 and not batch:
            return [K.kes_krylov_solve(h, R0_dev[0], so)]
        return K.kes_block_krylov_solve(h, R0_dev, b, so)

    for _ in range(max(args.warmup, 0)):
        res = solve()
    K.kes_reset_stats(h)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(dist)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(args.steps):
                res = solve()
            e1.record(stream)
        torch.cuda.synchronize()
    barrier(dist)
    ms_local = e0.elapsed_time(e1)
    stats = K.kes_get_stats(h)
    ms_total = max_over_ranks(dist, ms_local, dev)
    steps_per_solve = res[0]["time_steps"]
    units_local = n * b * steps_per_solve * args.steps
    units = sum_over_ranks(dist, units_local, dev)
    value = units / (ms_total / 1e3) / 1e9

    # roofline of the fused step kernel, timed by the library's CUDA events on its stream
    step_ms = stats["filter_ms"] / max(stats["filter_steps"], 1)
    bytes_step = K.kes_step_bytes(h, b, 1)
    achieved = bytes_step / (step_ms / 1e3) / 1e9
    peak, peak_src = load_peak()
    traffic = profiled_traffic(args.workload, STEP_KERNEL_SRC if b == 1 else BLOCK_KERNEL_SRC)

    # several intervals from one trajectory: the same block filtered with F weight tables
    multi = None
    if F > 1:
        K.kes_set_filters_batch(h, wmin_all, wmax_all, taus, wl.L)
        out = torch.zeros((F, b, n), dtype=torch.float64, device=dev)
        K.kes_filter_apply(h, R0_dev, out, b)
        K.kes_sync(h)
        K.kes_reset_stats(h)
        reps = 3
        for _ in range(reps):
            K.kes_filter_apply(h, R0_dev, out, b)
        st = K.kes_get_stats(h)
        fms = st["filter_ms"] / reps
        bF = K.kes_step_bytes(h, b, F)
        multi = {"F": F, "b": b, "L": wl.L, "ms_per_filter": fms,
                 "value": n * b * wl.L / (fms / 1e3) / 1e9, "unit": METRIC,
                 "step_us": 1e3 * fms / wl.L, "achieved_gbs": bF / (fms / wl.L / 1e3) / 1e9,
                 "algorithmic_bytes_per_step": bF}
        K.kes_set_filters_batch(h, wmin1, wmax1, taus, wl.L)

    # end to end through the C ABI with host buffers: start block from pinned memory in,
    # accepted Ritz pairs (values and vectors) out, every step
    R0_pinned = torch.from_numpy(R0_host).pin_memory()
    so_e2e = K.kes_solve_opts_default()
    so_e2e.kmax, so_e2e.tol, so_e2e.want_vectors, so_e2e.check_every = so.kmax, so.tol, 1, so.check_every
    e2e_steps = args.e2e_steps
    barrier(dist)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out_bytes = 0
    r = res
    for _ in range(e2e_steps):
        if b == 1 and not batch:
            r = [K.kes_krylov_solve(h, R0_pinned.numpy()[0], so_e2e)]
        else:
            r = K.kes_block_krylov_solve(h, R0_pinned.numpy(), b, so_e2e)
        out_bytes = sum((x["vectors"].nbytes if x["vectors"] is not None else 0) + 4 * x["n_pairs"] * 8 for x in r)
    torch.cuda.synchronize()
    e2e = None
    if e2e_steps > 0:
        e2e_s = max_over_ranks(dist, (time.perf_counter() - t0) / e2e_steps, dev)
        e2e = {"value": sum_over_ranks(dist, n * b * r[0]["time_steps"], dev) / e2e_s / 1e9, "unit": METRIC,
               "h2d_bytes_per_step": 8 * n * b, "d2h_bytes_per_step": out_bytes}

    # accuracy of the accepted pairs against the exact spectrum (tensor grids)
    eig_err = None
    for p, rr, iv in zip(problems, res, ivs):
        if p.cells and not p.meta.get("length") and rr["n_pairs"]:
            for t, f in zip(rr["omega2"], rr["interval"]):
                exact = spectra.omega2_in(p.cells, p.h, iv[f][0], iv[f][1])
                e = float(np.min(np.abs(exact - t)) / t)
                eig_err = e if eig_err is None else max(eig_err, e)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        big = max(range(len(problems)), key=lambda j: problems[j].n)
        v, steps, dt = oracle_sample(problems[big], taus[big], wl, args.cpu_seconds, ivs[big][0])
        cpu = {"value": v, "unit": METRIC, "cores": cpu_cores_used(), "kind": "oracle",
               "sample": f"{steps} leapfrog steps of the FP64 oracle filter, one vector, on "
                         f"{problems[big].name} ({problems[big].n} dofs, {dt:.1f} s)"}

    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if wl.precision == "fp64" else "f32",
        "data": "synthetic",
        "config": {"workload": args.workload, "meshes": len(problems), "dofs": n, "nnz": nnz, "b": b,
                   "interval": ([float(wmin1[0, 0]), float(wmax1[0, 0])] if not batch
                                else f"per mesh, {F_solve} interval(s) with {b // F_solve} column(s) each"),
                   "L": wl.L, "kmax": wl.kmax, "tau": float(taus[0]) if not batch else "per mesh",
                   "omega_max_power": float(omega_pow[0]) if not batch else "per mesh",
                   "format": "SELL-32 (sigma=1)", "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (matrix > 129 MB)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_source": peak_src,
                     "kernel": ("k_step_f64" if wl.precision == "fp64" else "k_step_f32") if b == 1
                     else ("k_step_blk<double>" if wl.precision == "fp64" else "k_step_blk<float>"),
                     "step_variant": stats["step_variant"] if b == 1 else stats["blk_variant"],
                     "step_grid": stats["step_grid"] if b == 1 else stats["blk_grid"],
                     "step_us": step_ms * 1e3, "algorithmic_bytes_per_step": bytes_step},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(stats["kernel_launches"]),
        "clocks": clk.summary(),
        "solve": {"accepted_pairs": [x["n_pairs"] for x in res] if batch else res[0]["n_pairs"],
                  "k_used": res[0]["k_used"], "time_steps": steps_per_solve,
                  "max_rel_res": max((float(x["rel_res"].max()) for x in res if x["n_pairs"]), default=None),
                  "max_eig_rel_err_vs_exact": eig_err, "filter_ms_share": stats["filter_ms"] / ms_local,
                  "other_kernels_ms_share": stats["solve_other_ms"] / ms_local},
    }
    if multi:
        line["filter_multi_interval"] = multi
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- reference arm

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle as O
    from fe_inputs import WORKLOADS
    wl = WORKLOADS[args.workload]
    problems, _ = workload_problems(wl)
    big = max(range(len(problems)), key=lambda j: problems[j].n)
    problem = problems[big]
    iv = wl.mesh_intervals(problem)[0]
    S = problem.to_scipy()
    omega_pow = O.power_iteration(S, problem.m, start_block([problem], 1, wl.seed)[0], wl.power_iters)
    tau = wl.cfl * 2.0 / omega_pow
    per_step_budget = max(1.0, 60.0 / max(args.steps + args.warmup, 1))
    samples = []
    for i in range(args.warmup + args.steps):
        v, steps, dt = oracle_sample(problem, tau, wl, per_step_budget, iv)
        if i >= args.warmup:
            samples.append((v, steps, dt))
    total_units = sum(problem.n * s for _, s, _ in samples)
    total_s = sum(dt for _, _, dt in samples)
    value = total_units / total_s / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / max(len(samples), 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "dofs": problem.n, "nnz": problem.nnz,
                   "interval": list(iv), "L": wl.L, "kmax": wl.kmax, "tau": tau},
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": cpu_cores_used(), "kind": "oracle",
                         "sample": f"each step = {samples[0][1] if samples else 0} leapfrog steps of the FP64 "
                                   f"oracle filter on {problem.name}"},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


TTS_FORMS = (
    # name, precision, block width, FP64 refinement sweeps, refinement filter length / L
    ("fp64", "fp64", 1, 0, 1.0),
    ("fp32+refine1", "fp32", 1, 1, 1.0),
    ("fp32+refine1_L/4", "fp32", 1, 1, 0.25),
    ("fp32+refine1_L/8", "fp32", 1, 1, 0.125),
)
TTS_KMAX = (160, 200, 240, 280, 320, 360, 400)   # coarse sweep; then steps of 10 below the first success


def run_tts(args):
    """Time to all eigenpairs in the interval at rel_res <= 1e-8, on the 128^3 cube
    (eigenvalues of multiplicity up to 6) and on a box of the same size with simple
    eigenvalues: for each form a sweep over the Krylov dimension kmax (one projection at
    the end, so that every run costs what a solve of that size costs), reporting each
    run's time and the distinct eigenvalues it accepted; a form's time to solution is
    that of the smallest kmax (to within 10) that accepts every distinct eigenvalue.
    The FP32 forms reach 1e-8 through FP64 refinement sweeps on their in-interval Ritz
    vectors, filtered 8 at a time, with the full filter or its first L/4 or L/8 steps."""
    import numpy as np
    import torch

    import paper_2402_08515_gb300 as K
    from fe_inputs import WORKLOADS, start_vectors
    from fe_inputs import spectra

    tol = 1e-8
    forms = [f for f in TTS_FORMS if not args.tts_forms or f[0] in args.tts_forms.split(",")]
    out = []
    for wname in args.tts_workloads.split(","):
        wl = WORKLOADS[wname]
        p = wl.build()
        exact = spectra.omega2_in(p.cells, p.h, wl.omega_min, wl.omega_max)
        distinct, _ = spectra.cluster(exact)
        v0 = start_vectors(p.n, 1, wl.seed)[0]
        runs, summary = [], {}
        for name, prec, b, refine, frac in forms:
            summary[name] = None
            with K.Context(p, precision=prec, block_b=8) as c:
                w, _ = K.kes_estimate_omega_max(c.handle, wl.power_iters, v0)
                K.kes_set_filter(c.handle, wl.omega_min, wl.omega_max, wl.cfl * 2 / w, wl.L)
                R = start_vectors(p.n, b, wl.seed + 1)

                def run(kmax):
                    so = K.kes_solve_opts_default()
                    so.kmax, so.tol, so.check_every, so.refine_sweeps = kmax, tol, kmax, refine
                    so.refine_L = int(round(frac * wl.L)) if frac < 1.0 else 0
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    res = K.kes_block_krylov_solve(c.handle, R, b, so)[0]
                    dt = time.perf_counter() - t0
                    found, _ = spectra.cluster(res["omega2"])
                    err = max((float(np.min(np.abs(exact - t)) / t) for t in res["omega2"]), default=None)
                    runs.append({"form": name, "b": b, "kmax": kmax, "refine_sweeps": refine,
                                 "refine_L": so.refine_L or wl.L, "seconds": dt,
                                 "accepted_pairs": res["n_pairs"], "accepted_distinct": len(found),
                                 "max_rel_res": float(res["rel_res"].max()) if res["n_pairs"] else None,
                                 "max_eig_rel_err_vs_exact": err, "leapfrog_steps": res["time_steps"],
                                 "fp64_refine_steps": res["refine_steps"]})
                    print(json.dumps({"workload": wname, **runs[-1]}), file=sys.stderr, flush=True)
                    if len(found) >= len(distinct):
                        summary[name] = {"seconds": dt, "kmax": kmax, "accepted_pairs": res["n_pairs"]}
                        return True
                    return False

                last_fail = None
                for kmax in TTS_KMAX:
                    if run(kmax):
                        lo = (last_fail or kmax - 40) + 10
                        for k in range(lo, kmax, 10):   # the coarse step overshoots by up to 30
                            if run(k):
                                break
                        break
                    last_fail = kmax
        out.append({"workload": wname, "dofs": p.n, "interval": [wl.omega_min, wl.omega_max], "L": wl.L,
                    "distinct_in_interval": len(distinct), "eigenvalues_in_interval": len(exact),
                    "time_to_all_distinct": summary, "runs": runs})
    print(json.dumps({"mode": "tts", "tol": tol, "workloads": out}), flush=True)


def run_weights(args):
    """Weight functions compared on the 64^2 square (Sec. 4, "Weight function"): the
    indicator of [20, 30] against a Gaussian and a triangular band centred at 25 with
    half of their peak at the interval's ends. For each: the filter factor beta~ over
    the exact spectrum (smallest inside the interval, largest outside) and the FP64
    Krylov solve until every distinct eigenvalue of [20, 30] is accepted at 1e-8."""
    import math

    import numpy as np
    import torch

    import paper_2402_08515_gb300 as K
    from fe_inputs import WORKLOADS, start_vectors
    from fe_inputs import spectra

    wl = WORKLOADS["square64_fp64"]
    p = wl.build()
    lo, hi = wl.omega_min, wl.omega_max
    c0, half = 0.5 * (lo + hi), 0.5 * (hi - lo)
    w_all = np.sqrt(spectra.grid_omega2(p.cells, p.h))
    inside = (w_all >= lo) & (w_all <= hi)
    distinct, _ = spectra.cluster(spectra.omega2_in(p.cells, p.h, lo, hi))
    v0 = start_vectors(p.n, 1, wl.seed)[0]
    rows = []
    with K.Context(p, precision="fp64") as c:
        w, _ = K.kes_estimate_omega_max(c.handle, wl.power_iters, v0)
        tau = wl.cfl * 2 / w
        L = wl.L
        tables = {
            "indicator": K.kes_alpha_table(lo, hi, tau, L),
            "gaussian": K.kes_alpha_gaussian(c0, half / math.sqrt(2 * math.log(2)), tau, L),
            "triangle": K.kes_alpha_triangle(c0, 2 * half, tau, L),
        }
        for name, alpha in tables.items():
            beta = K.kes_weights_response(alpha, tau, w_all)
            K.kes_set_weights(c.handle, alpha[None, None, :], [[lo]], [[hi]], [tau], L)
            # the smallest Krylov dimension (steps of 5) that accepts every distinct eigenvalue
            for kmax in range(20, 305, 5):
                so = K.kes_solve_opts_default()
                so.kmax, so.tol, so.check_every = kmax, 1e-8, kmax
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                res = K.kes_krylov_solve(c.handle, start_vectors(p.n, 1, wl.seed + 1)[0], so)
                dt = time.perf_counter() - t0
                found, _ = spectra.cluster(res["omega2"])
                if len(found) >= len(distinct):
                    break
            rows.append({"weight": name, "beta_min_inside": float(np.abs(beta[inside]).min()),
                         "beta_max_outside": float(np.abs(beta[~inside]).max()),
                         "accepted_distinct": len(found), "distinct_in_interval": len(distinct),
                         "krylov_vectors": res["k_used"], "leapfrog_steps": res["time_steps"], "seconds": dt})
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    print(json.dumps({"mode": "weights", "workload": "square64", "interval": [lo, hi], "L": L, "tau": tau,
                      "tol": 1e-8, "runs": rows}), flush=True)


def main(argv=None):
    args = parse_args(argv)
    if args.mode == "tts":
        run_tts(args)
        return
    if args.mode == "weights":
        run_weights(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_kes(args)


if __name__ == "__main__":
    main()
