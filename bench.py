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
TTS_TOL = 1e-8
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
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--tts-repeats", type=int, default=3, help="timed converged solves of the tts field")
    ap.add_argument("--no-tts", action="store_true", help="leave out the converged solve (tts, and e2e through it)")
    ap.add_argument("--no-precision-compare", action="store_true",
                    help="leave out the FP32-form against FP64 time to converged pairs (box2m)")
    ap.add_argument("--no-batch-filter", action="store_true", help="leave out the 12-mesh batched filter measurement")
    ap.add_argument("--cpu-seconds", type=float, default=20.0, help="budget of the oracle samples (1 core + all cores)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mode", default="solve", choices=["solve", "filter", "tts", "weights", "certify"],
                    help="filter: one filter application only (small profiling runs); tts: time to "
                         "converged eigenpairs at residual 1e-8, FP64 form against the FP32 forms with FP64 "
                         "refinement")
    ap.add_argument("--tts-forms", default="", help="comma-separated subset of the --mode tts forms")
    ap.add_argument("--tts-kmax", default="", help="comma-separated Krylov dimensions: run each form at these only "
                                                   "(no search)")
    ap.add_argument("--tts-workloads", default="cube128_fp64,box2m_fp64", help="workloads of --mode tts")
    ap.add_argument("--L", type=int, default=0, help="override the workload's time steps (--mode filter, certify)")
    ap.add_argument("--kmax", type=int, default=0, help="override the workload's Krylov dimension (--mode certify)")
    ap.add_argument("--interval", default="", help="override the filter interval as 'wmin,wmax' (--mode certify)")
    ap.add_argument("--tol", type=float, default=0.0, help="override the acceptance tolerance (--mode solve, certify)")
    ap.add_argument("--refine-sweeps", type=int, default=0, help="FP64 refinement sweeps (--mode solve, certify)")
    ap.add_argument("--refine-extra", type=int, default=0,
                    help="buffer Ritz vectors of the refinement (--mode solve, certify)")
    ap.add_argument("--refine-x2", action="store_true",
                    help="refinement filter in FP32 pairs instead of FP64 (--mode solve, certify; FP32 form)")
    ap.add_argument("--precision", default="", choices=["", "fp64", "fp32"],
                    help="override the workload's precision (--mode certify)")
    ap.add_argument("--b", type=int, default=0, help="override the workload's block width (--mode certify)")
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
    """Hash of the kernel source without its // comments and blank lines: a profile
    stays valid across comment edits and goes stale when any code changes."""
    code = []
    for line in open(src, encoding="utf-8").read().splitlines():
        line = re.sub(r"//.*$", "", line).strip()
        if line:
            code.append(line)
    return hashlib.sha256("\n".join(code).encode()).hexdigest()[:16]


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


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part", "hardware")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


# The all-core baseline: P processes (spawned: the parent holds a CUDA context) each run
# the oracle's filter, as it stands, on the same matrix, mapped read-only from .npy files
# so that the processes share one copy. Every process takes one job per round and waits
# on a barrier of P parties before it starts, so the P samples of a round run at once.
def _oracle_worker(path, barrier, jobs, results):
    import numpy as np
    import scipy.sparse as sp

    import oracle as O
    d = {k: np.load(os.path.join(path, k + ".npy"), mmap_mode="r")
         for k in ("row_ptr", "col", "val", "m", "r")}
    n = d["m"].shape[0]
    S = sp.csr_matrix((d["val"], d["col"], d["row_ptr"]), shape=(n, n), copy=False)
    m, r = np.array(d["m"]), np.array(d["r"])
    while True:
        job = jobs.get()
        if job is None:
            return
        tau, wmin, wmax, steps = job
        alpha = O.alpha_table(wmin, wmax, tau, steps)
        barrier.wait(timeout=600)
        t0 = time.time()
        out = O.filter_apply(S, m, r, tau, alpha)
        t1 = time.time()
        results.put((n * steps, t0, t1, bool(np.isfinite(out).all())))


class OraclePool:
    """P oracle processes over one matrix; round(steps) runs `steps` leapfrog steps of the
    oracle filter in every process at once and returns (dof-steps, wall seconds)."""

    def __init__(self, problem, r, tau, interval, procs: int):
        import multiprocessing as mp
        import numpy as np
        self.n_procs, self.tau, self.interval = procs, tau, interval
        base = "/dev/shm" if os.path.isdir("/dev/shm") else None
        self.dir = tempfile.mkdtemp(prefix="kes_oracle_", dir=base)
        for k, a in (("row_ptr", problem.row_ptr.astype(np.int64)), ("col", problem.col.astype(np.int64)),
                     ("val", problem.val), ("m", problem.m), ("r", r)):
            np.save(os.path.join(self.dir, k + ".npy"), np.ascontiguousarray(a))
        ctx = mp.get_context("spawn")
        self.jobs = [ctx.Queue() for _ in range(procs)]
        self.results = ctx.Queue()
        self.barrier = ctx.Barrier(procs)      # kept alive while the processes use it
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in saved:
            os.environ[k] = "1"
        try:
            self.procs = [ctx.Process(target=_oracle_worker, args=(self.dir, self.barrier, q, self.results),
                                      daemon=True)
                          for q in self.jobs]
            for pr in self.procs:
                pr.start()
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def round(self, steps: int, timeout: float = 900.0):
        import queue
        job = (self.tau, self.interval[0], self.interval[1], int(steps))
        for q in self.jobs:
            q.put(job)
        out, t_end = [], time.time() + timeout
        while len(out) < self.n_procs:
            try:
                out.append(self.results.get(timeout=1.0))
            except queue.Empty:
                if time.time() > t_end or not all(pr.is_alive() for pr in self.procs):
                    raise RuntimeError("an oracle process ended or timed out")
        assert all(ok for *_, ok in out)
        return sum(u for u, *_ in out), max(t1 for _, _, t1, _ in out) - min(t0 for _, t0, _, _ in out)

    def close(self):
        import shutil
        for q in self.jobs:
            q.put(None)
        for pr in self.procs:
            pr.join(timeout=30)
            if pr.is_alive():
                pr.terminate()
        shutil.rmtree(self.dir, ignore_errors=True)


def small_solve_oracle(small: dict | None) -> dict | None:
    """The oracle's whole eigensolve (Algorithm 2.5 with the same start vector, tau and
    sizes) on the small case the GPU solved (small_solve_gpu), in one process."""
    if not small:
        return None
    import numpy as np
    import oracle as O
    from fe_inputs import WORKLOADS, start_vectors
    wl = WORKLOADS[small["workload"]]
    p = wl.build()
    r0 = start_vectors(p.n, 1, wl.seed + 1)[0]
    t0 = time.perf_counter()
    res = O.krylov_solve(p.to_scipy(), p.m, r0, wl.omega_min, wl.omega_max, small["tau"], wl.L, wl.kmax, 1e-8,
                         check_every=wl.check_every, keep_basis=False)
    dt = time.perf_counter() - t0
    gpu = np.asarray(small["gpu_omega2"])
    # pairs near the acceptance threshold may be accepted on one side only; the ones both
    # accept (within 1e-10) are compared
    diffs = [float(np.min(np.abs(res.omega2 - t)) / t) for t in gpu] if res.omega2.size else []
    common = [d for d in diffs if d <= 1e-10]
    out = {k: v for k, v in small.items() if k != "gpu_omega2"}
    out.update(oracle_s=dt, oracle_cores=1, oracle_accepted=int(res.omega2.size),
               accepted_by_both=len(common),
               max_rel_diff_of_pairs_both_accept=max(common, default=None),
               gpu_accepted_omega=[float(np.sqrt(t)) for t in gpu],
               oracle_accepted_omega=[float(w) for w in res.omega])
    return out


def cpu_baseline(problem, tau, wl, seconds: float, interval, small: dict | None = None) -> dict:
    """The oracle on the host cores: one process (single core) and P processes (all cores),
    each a bounded sample of the workload's filter; and the oracle's whole solve of the
    small case beside the GPU's."""
    from fe_inputs import start_vectors
    v1, steps1, dt1 = oracle_sample(problem, tau, wl, seconds / 2, interval)
    P = host_cores()
    per_step = dt1 / steps1
    pool = OraclePool(problem, start_vectors(problem.n, 1, wl.seed)[0], tau, interval, P)
    try:
        pool.round(2)                                          # maps the matrix in every process
        steps = int(max(3, min(wl.L, seconds / 2 / per_step)))
        units, wall = pool.round(steps)
    except Exception as e:                                     # report the one-core figure alone
        return {"value": v1, "unit": METRIC, "cores": 1, "kind": "oracle",
                "sample": f"{steps1} leapfrog steps of the FP64 oracle filter in one process, {dt1:.1f} s",
                "all_cores_error": repr(e)[:200], "cpu_model": cpu_model()}
    finally:
        pool.close()
    return {"value": units / wall / 1e9, "unit": METRIC, "cores": P, "kind": "oracle",
            "sample": f"{P} processes, one per host core, each {steps} leapfrog steps of the FP64 oracle filter "
                      f"(one vector) on {problem.name} ({problem.n} dofs) at once, {wall:.1f} s wall",
            "small_case_solve": small_solve_oracle(small),
            "cpu_model": cpu_model(),
            "single_core": {"value": v1, "cores": 1,
                            "sample": f"{steps1} leapfrog steps of the same filter in one process, {dt1:.1f} s"}}


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

def precision_comparison(dev, stream) -> dict:
    """The FP32 form against plain FP64, time to every eigenpair of an interval at
    rel_res <= 1e-8 on a workload whose interval holds simple eigenvalues (box2m, [24, 28],
    81 of them): the FP64 single-vector solve at its Krylov dimension, and the FP32 solve
    followed by one refinement sweep of half length in FP32 pairs over its in-interval Ritz
    vectors (8 columns per SpMM step), each one solve on a fresh context with the input
    resident, CUDA events on the library stream around the synchronous call. The Krylov
    dimensions are those of `--mode tts` (the smallest that accept all 81, to within 10)."""
    import numpy as np
    import torch

    import paper_2402_08515_gb300 as K
    from fe_inputs import WORKLOADS, start_vectors
    from fe_inputs import spectra
    wl = WORKLOADS["box2m_fp64"]
    p = wl.build()
    exact = spectra.omega2_in(p.cells, p.h, wl.omega_min, wl.omega_max)
    distinct, _ = spectra.cluster(exact)
    v0 = start_vectors(p.n, 1, wl.seed)[0]
    r0 = torch.from_numpy(start_vectors(p.n, 1, wl.seed + 1)[0]).to(dev)
    forms = (("fp64", "fp64", 1, wl.tts_kmax, 0, 0, K.KES_REFINE_FP64),
             ("fp32+refine1x2_L/2", "fp32", 8, 240, 1, wl.L // 2, K.KES_REFINE_F32X2))
    out = {"workload": "box2m_fp64", "dofs": p.n, "interval": [wl.omega_min, wl.omega_max], "L": wl.L,
           "tol": TTS_TOL, "distinct_in_interval": len(distinct), "forms": {}}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index or 0) as clk:
        for name, prec, bb, kmax, sweeps, refine_L, rprec in forms:
            with K.Context(p, precision=prec, stream=stream, block_b=bb) as ctx:
                h = ctx.handle
                w, _ = K.kes_estimate_omega_max(h, wl.power_iters, v0)
                K.kes_set_filter(h, wl.omega_min, wl.omega_max, wl.cfl * 2 / w, wl.L)
                so = K.kes_solve_opts_default()
                so.kmax, so.tol, so.check_every = kmax, TTS_TOL, kmax
                so.refine_sweeps, so.refine_L, so.refine_precision = sweeps, refine_L, rprec
                torch.cuda.synchronize()
                with torch.cuda.stream(stream):
                    e0.record(stream)
                    res = K.kes_krylov_solve(h, r0, so)
                    e1.record(stream)
                torch.cuda.synchronize()
                found, _ = spectra.cluster(res["omega2"])
                out["forms"][name] = {
                    "seconds": e0.elapsed_time(e1) / 1e3, "kmax": kmax, "refine_sweeps": sweeps,
                    "refine_L": refine_L, "refine_precision": ("fp64", "fp32x2")[rprec],
                    "accepted_pairs": res["n_pairs"], "accepted_distinct": len(found),
                    "all_distinct_found": len(found) >= len(distinct),
                    "max_rel_res": float(res["rel_res"].max()) if res["n_pairs"] else None,
                    "max_eig_rel_err_vs_exact": max((float(np.min(np.abs(exact - t)) / t) for t in res["omega2"]),
                                                    default=None)}
    f64, f32 = out["forms"]["fp64"], out["forms"]["fp32+refine1x2_L/2"]
    out["fp64_over_fp32_time"] = f64["seconds"] / f32["seconds"]
    out["clocks"] = clk.summary()
    return out


def batch_filter_measurement(dev, stream, reps: int = 3) -> dict:
    """The batched SpMM step on the 12-mesh batch (3.14 M dofs, 8 FP32 columns per mesh, one
    interval per mesh; and the four intervals of every mesh from one trajectory): one filter
    application of L = 600 steps, warm, then `reps` timed by the library's CUDA events."""
    import numpy as np
    import torch

    import paper_2402_08515_gb300 as K
    from fe_inputs import WORKLOADS
    wl = WORKLOADS["batch12_fp32"]
    problems = wl.build()
    n = sum(p.n for p in problems)
    out = {"workload": "batch12_fp32", "meshes": len(problems), "dofs": n, "b": wl.b, "L": wl.L}
    peak, _ = load_peak()
    with K.Context(problems, precision=wl.precision, stream=stream, block_b=wl.b) as ctx:
        h = ctx.handle
        omega, _ = K.kes_estimate_omega_max_batch(h, wl.power_iters, start_block(problems, 1, wl.seed)[0])
        taus = wl.cfl * 2.0 / omega
        ivs = [wl.mesh_intervals(p) for p in problems]
        R = torch.from_numpy(start_block(problems, wl.b, wl.seed + 1)).to(dev)
        for F in (1, len(ivs[0])):
            wmin = np.array([[a for a, _ in iv[:F]] for iv in ivs])
            wmax = np.array([[c for _, c in iv[:F]] for iv in ivs])
            K.kes_set_filters_batch(h, wmin, wmax, taus, wl.L)
            res = torch.zeros((F, wl.b, n), dtype=torch.float64, device=dev)
            K.kes_filter_apply(h, R, res, wl.b)
            K.kes_sync(h)
            K.kes_reset_stats(h)
            for _ in range(reps):
                K.kes_filter_apply(h, R, res, wl.b)
            st = K.kes_get_stats(h)
            step_us = 1e3 * st["filter_ms"] / max(st["filter_steps"], 1)
            nbytes = K.kes_step_bytes(h, wl.b, F)
            gbs = nbytes / (step_us / 1e6) / 1e9
            out[f"F{F}"] = {"step_us": step_us, "algorithmic_bytes_per_step": nbytes, "achieved_gbs": gbs,
                            "frac": gbs / peak, "gdof_steps_per_s": n * wl.b / (step_us / 1e6) / 1e9,
                            "finite": bool(torch.isfinite(res).all())}
        out["kernel"] = "k_step_blk<float,8>"
        out["blk_variant"] = st["blk_variant"]
        out["timing"] = f"{reps} filter applications of {wl.L} steps, CUDA events on the library stream, after one warm"
    return out


def small_solve_gpu(stream) -> dict:
    """The small case (64^2 square, [20, 30], L = 300, Krylov dimension 40, FP64) solved on
    the GPU: wall time of the call, accepted pairs (compared with the oracle's solve of the
    same problem in the CPU baseline)."""
    import torch

    import paper_2402_08515_gb300 as K
    from fe_inputs import WORKLOADS, start_vectors
    wl = WORKLOADS["square64_fp64"]
    p = wl.build()
    with K.Context(p, precision="fp64", stream=stream) as c:
        w, _ = K.kes_estimate_omega_max(c.handle, wl.power_iters, start_vectors(p.n, 1, wl.seed)[0])
        tau = wl.cfl * 2.0 / w
        K.kes_set_filter(c.handle, wl.omega_min, wl.omega_max, tau, wl.L)
        so = K.kes_solve_opts_default()
        so.kmax, so.tol, so.check_every = wl.kmax, 1e-8, wl.check_every
        r0 = start_vectors(p.n, 1, wl.seed + 1)[0]
        K.kes_krylov_solve(c.handle, r0, so)                    # warm
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = K.kes_krylov_solve(c.handle, r0, so)
        dt = time.perf_counter() - t0
    return {"workload": "square64_fp64", "dofs": p.n, "kmax": wl.kmax, "L": wl.L, "tau": tau,
            "gpu_s": dt, "gpu_accepted": res["n_pairs"], "gpu_omega2": [float(t) for t in res["omega2"]]}


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
    so.kmax, so.tol, so.check_every = wl.kmax, args.tol or wl.acceptance(), wl.check_every
    so.refine_sweeps, so.refine_extra = args.refine_sweeps, args.refine_extra
    so.refine_precision = K.KES_REFINE_F32X2 if args.refine_x2 else K.KES_REFINE_FP64
    R0_host = start_block(problems, b, wl.seed + 1 + 1000 * rank)
    R0_dev = torch.from_numpy(R0_host).to(dev)
    torch.cuda.synchronize()
    if args.mode == "filter":
        L = args.L or wl.L
        K.kes_set_filters_batch(h, wmin1[:, :1], wmax1[:, :1], taus, L)
        out = torch.zeros((1, b, n), dtype=torch.float64, device=dev)
        K.kes_filter_apply(h, R0_dev, out, b)      # the first application also captures the graph
        K.kes_sync(h)
        K.kes_reset_stats(h)
        K.kes_filter_apply(h, R0_dev, out, b)
        K.kes_sync(h)
        st = K.kes_get_stats(h)
        if rank == 0:
            print(json.dumps({"mode": "filter", "workload": args.workload, "L": L, "dofs": n, "b": b,
                              "filter_ms": st["filter_ms"], "step_us": 1e3 * st["filter_ms"] / L,
                              "step_variant": st["step_variant"], "blk_variant": st["blk_variant"],
                              "timing": "the second of two filter applications, CUDA events on the library stream",
                              "finite": bool(torch.isfinite(out).all())}))
        ctx.close()
        return

    def solve_with(opts):
        if b == 1 and not batch:
            return [K.kes_krylov_solve(h, R0_dev[0], opts)]
        return K.kes_block_krylov_solve(h, R0_dev, b, opts)

    def solve():
        return solve_with(so)

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

    # time to all eigenpairs of the interval at rel_res <= 1e-8: the FP64 solve at the Krylov
    # dimension that accepts every distinct eigenvalue of the interval (one projection, at the
    # end), inputs resident, CUDA events on the library's stream
    tts = None
    so_t = None
    if wl.tts_kmax and not batch and b == 1 and not args.no_tts:
        so_t = K.kes_solve_opts_default()
        so_t.kmax, so_t.tol, so_t.check_every = wl.tts_kmax, TTS_TOL, wl.tts_kmax
        res_t = solve_with(so_t)                                   # warm-up: sizes the basis
        times = []
        barrier(dist)
        torch.cuda.synchronize()
        with ClockSampler(local) as clk_t:
            for _ in range(max(1, args.tts_repeats)):
                with torch.cuda.stream(stream):
                    e0.record(stream)
                    res_t = solve_with(so_t)
                    e1.record(stream)
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1) / 1e3)
        barrier(dist)
        exact = spectra.omega2_in(problems[0].cells, problems[0].h, wmin1[0, 0], wmax1[0, 0])
        distinct, _ = spectra.cluster(exact)
        found, _ = spectra.cluster(res_t[0]["omega2"])
        t_med = max_over_ranks(dist, statistics.median(times), dev)
        tts = {"value": t_med, "unit": "s", "higher_is_better": False, "repeats_s": times,
               "kmax": wl.tts_kmax, "tol": TTS_TOL, "L": wl.L, "time_steps": res_t[0]["time_steps"],
               "accepted_pairs": res_t[0]["n_pairs"], "accepted_distinct": len(found),
               "distinct_in_interval": len(distinct), "eigenvalues_in_interval": len(exact),
               "all_distinct_found": len(found) >= len(distinct),
               "max_rel_res": float(res_t[0]["rel_res"].max()) if res_t[0]["n_pairs"] else None,
               "max_eig_rel_err_vs_exact": max((float(np.min(np.abs(exact - t)) / t) for t in res_t[0]["omega2"]),
                                               default=None),
               "gdof_steps_per_s": sum_over_ranks(dist, n * res_t[0]["time_steps"], dev) / t_med / 1e9,
               "kmax_source": "the smallest Krylov dimension (steps of 10) at which this solve, and the "
                              "solve 10 vectors larger, accept every distinct eigenvalue of the interval "
                              "(bench.py --mode tts)",
               "clocks": clk_t.summary()}

    # end to end through the C ABI with host buffers: start block from pinned memory in,
    # accepted Ritz pairs (values and vectors) out, every step; the converged solve when
    # the workload has one, else the headline solve
    R0_pinned = torch.from_numpy(R0_host).pin_memory()
    so_e2e = K.kes_solve_opts_default()
    src = so_t if so_t is not None else so
    so_e2e.kmax, so_e2e.tol, so_e2e.check_every, so_e2e.want_vectors = src.kmax, src.tol, src.check_every, 1
    so_e2e.refine_sweeps, so_e2e.refine_extra = src.refine_sweeps, src.refine_extra
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
        out_bytes = sum((x["vectors"].nbytes if x["vectors"] is not None else 0) + 4 * x["n_pairs"] * 8
                        + 4 * x["n_pairs"] for x in r)
    torch.cuda.synchronize()
    e2e = None
    if e2e_steps > 0:
        e2e_s = max_over_ranks(dist, (time.perf_counter() - t0) / e2e_steps, dev)
        e2e = {"value": sum_over_ranks(dist, n * b * r[0]["time_steps"], dev) / e2e_s / 1e9, "unit": METRIC,
               "h2d_bytes_per_step": 8 * n * b, "d2h_bytes_per_step": out_bytes,
               "solve": ("the converged solve of `tts` (kmax %d)" % so_e2e.kmax) if so_t is not None
                        else "the timed solve", "seconds_per_step": e2e_s,
               "accepted_pairs_returned": sum(x["n_pairs"] for x in r)}

    # accuracy of the accepted pairs against the exact spectrum (tensor grids)
    eig_err = None
    for p, rr, iv in zip(problems, res, ivs):
        if p.cells and not p.meta.get("length") and rr["n_pairs"]:
            for t, f in zip(rr["omega2"], rr["interval"]):
                exact = spectra.omega2_in(p.cells, p.h, iv[f][0], iv[f][1])
                e = float(np.min(np.abs(exact - t)) / t)
                eig_err = e if eig_err is None else max(eig_err, e)

    # the batched SpMM step of the 12-mesh batch (secondary: the default line's other kernel)
    batch_filter = None
    if args.workload == "cube128_fp64" and not args.no_batch_filter:
        batch_filter = batch_filter_measurement(dev, stream)

    # the FP32 form against plain FP64 to converged pairs at 1e-8 (simple eigenvalues)
    prec_cmp = None
    if args.workload == "cube128_fp64" and not args.no_precision_compare:
        prec_cmp = precision_comparison(dev, stream)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        big = max(range(len(problems)), key=lambda j: problems[j].n)
        small = small_solve_gpu(stream) if args.workload == "cube128_fp64" else None
        cpu = cpu_baseline(problems[big], taus[big], wl, args.cpu_seconds, ivs[big][0], small)

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
        "tts": tts,
        "precision_comparison": prec_cmp,
        "solve": {"tol": so.tol, "refine_sweeps": so.refine_sweeps, "refine_extra": so.refine_extra,
                  "refine_precision": ("fp64", "fp32x2")[so.refine_precision],
                  "accepted_pairs": [x["n_pairs"] for x in res] if batch else res[0]["n_pairs"],
                  "k_used": res[0]["k_used"], "time_steps": steps_per_solve,
                  "max_rel_res": max((float(x["rel_res"].max()) for x in res if x["n_pairs"]), default=None),
                  "max_eig_rel_err_vs_exact": eig_err, "filter_ms_share": stats["filter_ms"] / ms_local,
                  "other_kernels_ms_share": stats["solve_other_ms"] / ms_local},
    }
    if multi:
        line["filter_multi_interval"] = multi
    if batch_filter:
        line["batch12_filter"] = batch_filter
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- reference arm

def run_reference(args):
    """The oracle, as it stands, on every host core: one process per core, each step one
    bounded sample of the workload's filter in all of them at once (rank 0 only)."""
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
    v0 = start_block([problem], 1, wl.seed)[0]
    omega_pow = O.power_iteration(S, problem.m, v0, wl.power_iters)
    tau = wl.cfl * 2.0 / omega_pow
    P = host_cores()
    t0 = time.perf_counter()
    O.filter_apply(S, problem.m, v0, tau, O.alpha_table(iv[0], iv[1], tau, 3))
    per_step = (time.perf_counter() - t0) / 3
    # about 90 s of oracle work over all warm-up and timed steps
    steps = int(max(2, min(wl.L, 90.0 / max(args.steps + args.warmup, 1) / per_step)))
    pool = OraclePool(problem, v0, tau, iv, P)
    units, secs = 0, 0.0
    try:
        for i in range(args.warmup + args.steps):
            u, w = pool.round(steps)
            if i >= args.warmup:
                units += u
                secs += w
    finally:
        pool.close()
    value = units / secs / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "dofs": problem.n, "nnz": problem.nnz,
                   "interval": list(iv), "L": wl.L, "kmax": wl.kmax, "tau": tau},
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": P, "kind": "oracle", "cpu_model": cpu_model(),
                         "sample": f"each step = {steps} leapfrog steps of the FP64 oracle filter on {problem.name} "
                                   f"in each of {P} processes (one per host core) at once"},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


TTS_FORMS = (
    # name, precision, block width, refinement sweeps, refinement filter length / L, Ritz
    # vectors nearest outside the interval refined as a buffer, arithmetic of the refinement
    # filter (0 FP64, 1 FP32 pairs: the "x2" forms)
    ("fp64", "fp64", 1, 0, 1.0, 0, 0),
    ("fp32+refine1", "fp32", 1, 1, 1.0, 0, 0),
    ("fp32+refine1_L/2", "fp32", 1, 1, 0.5, 0, 0),
    ("fp32+refine1x2_L/2", "fp32", 1, 1, 0.5, 0, 1),
    ("fp64_b8", "fp64", 8, 0, 1.0, 0, 0),
    ("fp32_b8+refine1", "fp32", 8, 1, 1.0, 0, 0),
    ("fp32_b8+refine1+16", "fp32", 8, 1, 1.0, 16, 0),
    ("fp32_b8+refine1x2+16", "fp32", 8, 1, 1.0, 16, 1),
    ("fp32_b8+refine1_L/2", "fp32", 8, 1, 0.5, 0, 0),
    ("fp32_b8+refine1_L/2+16", "fp32", 8, 1, 0.5, 16, 0),
)
# coarse Krylov dimensions of the search (single vector, block of 8) and the final resolution
TTS_GRID = {1: (160, 200, 240, 280, 320, 360, 400), 8: (512, 640, 768, 896, 1024, 1152)}
TTS_RES = {1: 10, 8: 32}


def matched_pairs(exact, accepted) -> int:
    """Accepted Ritz values matched to the exact spectrum with multiplicity: for every
    distinct exact eigenvalue, min(multiplicity, accepted values within 1e-8 of it)."""
    import numpy as np
    from fe_inputs import spectra
    vals, mult = spectra.cluster(exact)
    acc = np.sort(np.asarray(accepted, dtype=np.float64))
    got = 0
    for v, m in zip(vals, mult):
        got += min(int(m), int(np.count_nonzero(np.abs(acc - v) <= 1e-8 * v)))
    return got


def run_tts(args):
    """Time to all eigenpairs in the interval at rel_res <= 1e-8, on the 128^3 cube
    (eigenvalues of multiplicity up to 6) and on a box of the same size with simple
    eigenvalues, for each form: the FP64 and FP32 single-vector solvers and the block
    solvers with b = 8 (Sec. 4, block version), the FP32 ones followed by one sweep of FP64
    filtered subspace iteration over their in-interval Ritz vectors (8 columns at a time,
    with the full filter or its first L/2 steps). A form's time to solution is that of the
    smallest Krylov dimension (one projection, at the end) that accepts every distinct
    eigenvalue of the interval, found by a coarse search and bisection; the block forms
    are also timed to every eigenpair with multiplicity. Runs that reach neither report
    the residual floor of their in-interval Ritz pairs."""
    import numpy as np
    import torch

    import paper_2402_08515_gb300 as K
    from fe_inputs import WORKLOADS, start_vectors
    from fe_inputs import spectra

    forms = [f for f in TTS_FORMS if not args.tts_forms or f[0] in args.tts_forms.split(",")]
    out = []
    with ClockSampler(0) as clk:
        for wname in args.tts_workloads.split(","):
            wl = WORKLOADS[wname]
            p = wl.build()
            exact = spectra.omega2_in(p.cells, p.h, wl.omega_min, wl.omega_max)
            distinct, _ = spectra.cluster(exact)
            v0 = start_vectors(p.n, 1, wl.seed)[0]
            runs, summary = [], {}
            for name, prec, b, refine, frac, extra, rprec in forms:
                with K.Context(p, precision=prec, block_b=8) as c:
                    w, _ = K.kes_estimate_omega_max(c.handle, wl.power_iters, v0)
                    K.kes_set_filter(c.handle, wl.omega_min, wl.omega_max, wl.cfl * 2 / w, wl.L)
                    R = start_vectors(p.n, b, wl.seed + 1)
                    cache = {}

                    def run(kmax):
                        if kmax in cache:
                            return cache[kmax]
                        so = K.kes_solve_opts_default()
                        so.kmax, so.tol, so.check_every, so.refine_sweeps = kmax, TTS_TOL, kmax, refine
                        so.refine_L = int(round(frac * wl.L)) if frac < 1.0 else 0
                        so.refine_extra, so.refine_precision = extra, rprec
                        K.kes_reset_stats(c.handle)
                        torch.cuda.synchronize()
                        t0 = time.perf_counter()
                        res = K.kes_block_krylov_solve(c.handle, R, b, so)[0]
                        dt = time.perf_counter() - t0
                        st = K.kes_get_stats(c.handle)
                        found, _ = spectra.cluster(res["omega2"])
                        inside = res["ritz_rel_res"][~np.isnan(res["ritz_rel_res"])]
                        rec = {"form": name, "b": b, "kmax": kmax, "refine_sweeps": refine, "refine_extra": extra,
                               "refine_precision": ("fp64", "fp32x2")[rprec],
                               "refine_L": so.refine_L or wl.L, "seconds": dt,
                               "accepted_pairs": res["n_pairs"], "accepted_distinct": len(found),
                               "matched_with_multiplicity": matched_pairs(exact, res["omega2"]),
                               "max_rel_res": float(res["rel_res"].max()) if res["n_pairs"] else None,
                               "ritz_rel_res_median_in_interval": float(np.median(inside)) if inside.size else None,
                               "max_eig_rel_err_vs_exact": max((float(np.min(np.abs(exact - t)) / t)
                                                                for t in res["omega2"]), default=None),
                               "leapfrog_steps": res["time_steps"], "refine_steps": res["refine_steps"],
                               "filter_s": st["filter_ms"] / 1e3, "other_kernels_s": st["solve_other_ms"] / 1e3}
                        runs.append(rec)
                        print(json.dumps({"workload": wname, **rec}), file=sys.stderr, flush=True)
                        cache[kmax] = rec
                        return rec

                    def search(ok):
                        """Smallest kmax (to TTS_RES[b]) of the grid's range with ok(run(kmax))."""
                        lo = None
                        for kmax in TTS_GRID[b]:
                            if ok(run(kmax)):
                                hi = kmax
                                lo = lo if lo is not None else max(b, kmax - (TTS_GRID[b][1] - TTS_GRID[b][0]))
                                while hi - lo > TTS_RES[b]:
                                    mid = (lo + hi) // 2 // b * b
                                    if mid <= lo or mid >= hi:
                                        break
                                    if ok(run(mid)):
                                        hi = mid
                                    else:
                                        lo = mid
                                r = run(hi)
                                return {"seconds": r["seconds"], "kmax": hi, "accepted_pairs": r["accepted_pairs"],
                                        "max_rel_res": r["max_rel_res"]}
                            lo = kmax
                        best = max(cache.values(), key=lambda r: r["accepted_distinct"])
                        return {"reached": False, "up_to_kmax": TTS_GRID[b][-1],
                                "best_accepted_distinct": best["accepted_distinct"],
                                "ritz_rel_res_median_in_interval": best["ritz_rel_res_median_in_interval"]}

                    if args.tts_kmax:                      # fixed Krylov dimensions, no search
                        for kmax in (int(t) for t in args.tts_kmax.split(",")):
                            run(kmax)
                        continue
                    summary[name] = {"all_distinct": search(lambda r: r["accepted_distinct"] >= len(distinct))}
                    if b > 1:
                        summary[name]["all_with_multiplicity"] = search(
                            lambda r: r["matched_with_multiplicity"] >= len(exact))
            out.append({"workload": wname, "dofs": p.n, "interval": [wl.omega_min, wl.omega_max], "L": wl.L,
                        "distinct_in_interval": len(distinct), "eigenvalues_in_interval": len(exact),
                        "time_to_solution": summary, "runs": runs})
    print(json.dumps({"mode": "tts", "tol": TTS_TOL, "clocks": clk.summary(), "workloads": out}), flush=True)


def run_certify(args):
    """One solve of the workload (block solver, every mesh) with the accepted Ritz vectors
    copied back, each pair certified on the host from its vector alone: the FP64 residual
    ||S x - theta M x||_2 / (theta ||M x||_2) of eq. (res) recomputed with the workload's
    CSR matrix (scipy), and, on tensor grids, the eigenvalue against the closed form."""
    import numpy as np
    import torch

    import paper_2402_08515_gb300 as K
    from fe_inputs import WORKLOADS
    from fe_inputs import spectra

    wl = WORKLOADS[args.workload]
    problems, batch = workload_problems(wl)
    b = args.b or wl.b
    precision = args.precision or wl.precision
    L = args.L or wl.L
    t_build = time.perf_counter()
    with K.Context(problems if batch else problems[0], precision=precision, block_b=b) as c:
        v0 = start_block(problems, 1, wl.seed)[0]
        omega_pow, _ = K.kes_estimate_omega_max_batch(c.handle, wl.power_iters, v0)
        taus = wl.cfl * 2.0 / omega_pow
        if args.interval:
            a, z = (float(t) for t in args.interval.split(","))
            ivs = [[(a, z)] for _ in problems]
        else:
            ivs = [wl.mesh_intervals(p)[:1] for p in problems]
        K.kes_set_filters_batch(c.handle, np.array([[iv[0][0]] for iv in ivs]), np.array([[iv[0][1]] for iv in ivs]),
                                taus, L)
        so = K.kes_solve_opts_default()
        so.kmax = args.kmax or wl.kmax
        so.tol = args.tol or (1e-8 if precision == "fp64" else wl.acceptance())
        so.check_every = so.kmax
        so.refine_sweeps = args.refine_sweeps
        so.refine_extra = args.refine_extra
        so.refine_precision = K.KES_REFINE_F32X2 if args.refine_x2 else K.KES_REFINE_FP64
        so.want_vectors = 1
        R0 = start_block(problems, b, wl.seed + 1)
        setup_s = time.perf_counter() - t_build
        torch.cuda.synchronize()
        with ClockSampler(0) as clk:
            t0 = time.perf_counter()
            res = K.kes_block_krylov_solve(c.handle, R0, b, so)
            solve_s = time.perf_counter() - t0
        meshes = []
        for p, r, iv, tau in zip(problems, res, ivs, taus):
            S = p.to_scipy()
            host_rel, eig_err = [], []
            for th, x in zip(r["omega2"], r["vectors"] if r["vectors"] is not None else []):
                mx = p.m * x
                host_rel.append(float(np.linalg.norm(S @ x - th * mx) / (th * np.linalg.norm(mx))))
                if p.cells and not p.meta.get("length"):
                    exact = spectra.omega2_in(p.cells, p.h, iv[0][0], iv[0][1])
                    eig_err.append(float(np.min(np.abs(exact - th)) / th) if exact.size else None)
            inside = r["ritz_rel_res"][~np.isnan(r["ritz_rel_res"])]
            meshes.append({"mesh": p.name, "dofs": p.n, "interval": list(iv[0]), "tau": float(tau),
                           "accepted_pairs": r["n_pairs"],
                           "omega": [float(w) for w in r["omega"]],
                           "library_rel_res_max": float(r["rel_res"].max()) if r["n_pairs"] else None,
                           "host_rel_res_max": max(host_rel) if host_rel else None,
                           "host_rel_res_all_within_tol": bool(all(h <= so.tol * (1 + 1e-6) for h in host_rel)),
                           "host_vs_library_rel_res_max_ratio": (max(h / l for h, l in zip(host_rel, r["rel_res"]))
                                                                 if host_rel else None),
                           "max_eig_rel_err_vs_exact": max((e for e in eig_err if e is not None), default=None),
                           "in_interval_ritz_values": int(inside.size),
                           "ritz_rel_res_median_in_interval": float(np.median(inside)) if inside.size else None,
                           "k_used": r["k_used"], "leapfrog_steps": r["time_steps"],
                           "refine_steps": r["refine_steps"]})
    print(json.dumps({"mode": "certify", "workload": args.workload, "precision": precision, "b": b, "L": L,
                      "kmax": so.kmax, "tol": so.tol, "refine_sweeps": so.refine_sweeps,
                      "refine_precision": ("fp64", "fp32x2")[so.refine_precision], "setup_s": setup_s,
                      "solve_s": solve_s, "clocks": clk.summary(), "meshes": meshes}), flush=True)


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
    if args.mode == "certify":
        run_certify(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_kes(args)


if __name__ == "__main__":
    main()
