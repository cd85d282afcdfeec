#!/usr/bin/env python
"""Hybrid IGA-ADS + CRVPINN time steps per second on one GB300 per rank.

Workload (one hybrid step, Sec. 6 of the paper): project the network pressure
into the B-spline space, CFL step size, 10 explicit saturation steps on a
256 x 256 quadratic C1 B-spline mesh (FP64), collocation coefficients, 100
Adam iterations of the CRVPINN robust loss on the 257 x 257 grid with a
2-64-64-64-64-1 tanh network (FP32).  Inputs are synthetic: a log-normal
permeability field (sigma 1, correlation length 0.1), Gaussian injector at
(0.25, 0.25) and producer at (0.75, 0.75), initial saturation 0.

Ranks run independent scenarios (weak scaling, no data-path collective).
`--impl reference` times the CPU oracle on the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("hybrid time steps/s (batched mixed-precision vs plain FP64) at stated error; "
          "p99 step ms")
UNIT = "steps/s"
FP32_LANES_PER_SM = 128
N_SM = 152
SM_MAX_MHZ = 2070.0


def args_parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--width", type=int, default=64)
    ap.add_argument("--adam-iters", type=int, default=100)
    ap.add_argument("--n-sub", type=int, default=10)
    ap.add_argument("--pretrain", type=int, default=6000)
    ap.add_argument("--base-iters", type=int, default=20000,
                    help="iterations of the base network every scenario starts from (0: Xavier start)")
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--scenarios", type=int, default=64)
    ap.add_argument("--streams", type=int, default=16)
    ap.add_argument("--assign", default="rr", choices=["rr", "lpt"],
                    help="scenarios to streams: balanced by estimated work, or round robin")
    ap.add_argument("--groups", type=int, default=2,
                    help="step the resident scenarios as this many batches (hybrid_step_batch: each "
                         "training kernel once per batch); 0: each scenario's own step on its stream")
    ap.add_argument("--budget-gb", type=float, default=8.0)
    ap.add_argument("--arrival-ms", type=float, default=20.0)
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--plain-steps", type=int, default=1)
    ap.add_argument("--c2-steps", type=int, default=20)
    ap.add_argument("--c1-steps", type=int, default=20)
    ap.add_argument("--large-steps", type=int, default=3)
    ap.add_argument("--err-iters", type=int, default=30000)
    ap.add_argument("--err-steps", type=int, default=3)
    ap.add_argument("--sat-n", type=int, default=4096)
    ap.add_argument("--only-degree", action="store_true",
                    help="only the degree-2/3/4 saturation-step leg")
    ap.add_argument("--degree-n", type=int, default=512,
                    help="mesh of the degree-2/3/4 FP64 saturation-step leg (0: skip)")
    ap.add_argument("--only-saturation", action="store_true",
                    help="run only the saturation-kernel block (a profiling aid) and print it")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-error", action="store_true", help="skip the stated-error measurement")
    ap.add_argument("--profile-iters", type=int, default=30)
    return ap.parse_args()


def workload_config(a, world, sizes=None):
    sizes = sizes or []
    mix = {n: sizes.count(n) for n in sorted(set(sizes))}
    return {
        "workload": f"{len(sizes)} resident scenarios per GPU, sizes {mix} (2D, p=2), FP32 "
                    f"saturation + CRVPINN 2-{a.width}x4-1 with BF16 tensor-core GEMMs (FP32 "
                    f"accumulate) on (n+1)^2 collocation; {a.n_sub} saturation steps + "
                    f"{a.adam_iters} Adam iterations per hybrid step; one step = one hybrid step "
                    f"of one scenario",
        "mlp": f"2-{a.width}x4-1", "ads_dtype": "f32", "crvpinn_dtype": "bf16 (tcgen05)",
        "n_sub": a.n_sub, "adam_iters": a.adam_iters, "lr": a.lr, "dt_policy": "cfl 0.1",
        "scenarios_per_gpu": len(sizes), "streams": a.streams, "stream_assignment": a.assign,
        "batches": (f"{a.groups} (hybrid_step_batch: grouped training launches)" if a.groups > 0
                    else "none (each scenario's own step graph on its stream)"),
        "parallelism": f"replicas x{world}",
        "rounds_timed": a.steps, "pretrain": a.pretrain,
        "network_start": (f"base network ({a.base_iters} iterations on K = 1, rate 1), output scaled by the "
                          "scenario's rate" if a.base_iters > 0 else "Xavier"),
        "l2": "working set of the resident mix exceeds L2 (129 MB); no flush",
    }


# ---------------------------------------------------------------------------
# distributed helpers (timing only: barrier and max over ranks)
# ---------------------------------------------------------------------------
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("BENCH_BACKEND", "nccl") == "nccl" else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world, device):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int, path=None):
        self.dev = device_index
        self.proc = None
        self.path = path
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.dev)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        if self.path:
            with open(self.path, "w") as f:
                f.write("\n".join(self.lines) + "\n")
        return clock_summary(self.lines)


def clock_summary(lines):
    """Median and maximum SM clock and the throttle reasons seen, from
    `nvidia-smi --query-gpu=<ClockSampler.FIELDS> --format=csv,noheader,nounits`
    lines; None if no line parses."""
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for ln in lines:
        parts = [p.strip() for p in ln.split(",")]
        if len(parts) < 9:
            continue
        try:
            sm.append(float(parts[1]))
            smax.append(float(parts[2]))
        except ValueError:
            continue
        for nm, v in zip(names, parts[5:9]):
            if v.lower().startswith("active"):
                reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
            "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# algorithmic work of the dominant kernels (per collocation point)
# ---------------------------------------------------------------------------
def mlp_flops_per_point(din, w):
    fwd = 2 * (din * w + 3 * w * w + w)
    bwd = 2 * (3 * 2 * w * w + w + din * w)
    return fwd, bwd


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def traffic_record(kernel):
    """DRAM bytes per launch from the committed ncu summary, if the kernel's
    source is unchanged since the capture (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        rec = json.load(f).get(kernel)
    if not rec:
        return None
    src = os.path.join(ROOT, rec["source"])
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()
    if h != rec.get("sha256"):
        return None
    return rec


# ---------------------------------------------------------------------------
# CPU oracle timing (the baseline and the reference arm)
#
# Each oracle hybrid step runs in a worker process of its own, started with
# `spawn` and with one BLAS/OpenMP thread (the oracle's scipy sparse LU and
# banded solves are single-threaded anyway), so `cores` is the number of
# workers that actually ran at once.
# ---------------------------------------------------------------------------
_SINGLE_THREAD_ENV = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def _oracle_step(job):
    """One oracle hybrid step of scenario `sc`: projection, CFL step size,
    `n_sub` saturation steps, then `measure` of the `adam_iters` Adam
    iterations (all of them when measure == adam_iters).  Returns the seconds
    of the non-network part, the seconds per measured Adam iteration, and the
    BLAS threads the worker ran with."""
    sc, n_sub, adam_iters, measure, lr, width = job
    from oracle.crvpinn import Adam
    from oracle.hybrid import HybridOracle
    from paper_2604_20731_gb300 import scenario as scn
    import numpy as np
    h = HybridOracle(sc, width=width)
    theta = scn.make_theta0(2, width, 4, seed=7)
    opt = Adam(theta.size)
    S = sc.S0_or_zero()
    h.crv.gram_solve_lu(np.zeros(h.crv.M))  # the Gram LU is factorised once (Eq. 28)
    t0 = time.perf_counter()
    P = h.project(theta)
    dt = h.ads.cfl_dt(P, cfl=0.1, dt_cap=1.0)
    for _ in range(n_sub):
        S = h.ads.step(S, P, dt)
    t1 = time.perf_counter()
    theta, _ = h.train(theta, opt, S, measure, lr)
    t2 = time.perf_counter()
    threads = None
    try:
        from threadpoolctl import threadpool_info
        threads = max([i.get("num_threads", 1) for i in threadpool_info()] or [1])
    except ImportError:
        threads = int(os.environ.get("OPENBLAS_NUM_THREADS", "0")) or None
    return t1 - t0, (t2 - t1) / max(measure, 1), threads


def _oracle_pool(workers):
    import multiprocessing as mp
    saved = {k: os.environ.get(k) for k in _SINGLE_THREAD_ENV}
    for k in _SINGLE_THREAD_ENV:
        os.environ[k] = "1"
    try:
        return mp.get_context("spawn").Pool(workers)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def oracle_baseline(a, mix, sizes):
    """CPU baseline for the GPU arm's line (rank 0): per mix size one oracle
    hybrid step, each single-threaded.  The non-network part is measured in
    full; of the Adam iterations 100 (128^2), 10 (256^2) and 3 (512^2) are
    measured and scaled to the step's count.  The scaling is checked on the
    128^2 member: its full step is also predicted from its first 2
    iterations.  The samples of the sizes run in parallel processes, but the
    figure is a single-threaded step rate."""
    picks = {n: mix[sizes.index(n)] for n in sorted(set(sizes))}
    measure = {n: (a.adam_iters if n <= 128 else (10 if n <= 256 else 3)) for n in picks}
    jobs = [(sc, a.n_sub, a.adam_iters, min(measure[n], a.adam_iters), a.lr, a.width) for n, sc in picks.items()]
    small = min(picks)
    jobs.append((picks[small], a.n_sub, a.adam_iters, 2, a.lr, a.width))
    with _oracle_pool(len(jobs)) as pool:
        res = pool.map(_oracle_step, jobs, chunksize=1)
    per_n = {n: r[0] + r[1] * a.adam_iters for n, r in zip(picks, res)}
    full = per_n[small]
    predicted = res[-1][0] + res[-1][1] * a.adam_iters
    mean_s = sum(per_n[n] for n in sizes) / len(sizes)
    threads = max([r[2] or 1 for r in res])
    return {"value": 1.0 / mean_s, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"one single-threaded oracle hybrid step per mix size, weighted by the mix: projection + "
                       f"CFL + {a.n_sub} saturation steps measured; Adam iterations measured "
                       f"{ {n: measure[n] for n in picks} } of {a.adam_iters} and scaled; the sizes' samples "
                       f"ran side by side in {len(jobs)} spawned single-threaded processes"),
            "seconds_per_step_by_n": per_n, "blas_threads_per_process": threads,
            "scaling_check": {"size": small, "full_step_s": full, "predicted_from_2_iterations_s": predicted,
                              "ratio": predicted / full}}


def run_reference(a, world, rank):
    """The oracle on the same mix: step k is one full hybrid step of mix
    member k (mod the mix) -- projection, CFL, the saturation steps and all
    Adam iterations, nothing extrapolated -- each in a single-threaded worker
    process; the steps run side by side on the host's cores."""
    if rank != 0:
        return 0
    mix = serving_mix(a.scenarios, seed=3)
    workers = max(1, min(os.cpu_count() or 1, a.steps))
    jobs = [(mix[k % len(mix)], a.n_sub, a.adam_iters, a.adam_iters, a.lr, a.width) for k in range(a.steps)]
    order = sorted(range(len(jobs)), key=lambda k: -jobs[k][0].n)  # largest first: balanced workers
    warm = scn_small(max(a.warmup, workers))
    with _oracle_pool(workers) as pool:
        pool.map(_oracle_step, [(sc, 1, 1, 1, a.lr, a.width) for sc in warm], chunksize=1)
        t0 = time.perf_counter()
        res = pool.map(_oracle_step, [jobs[k] for k in order], chunksize=1)
        wall = time.perf_counter() - t0
    value = a.steps / wall
    threads = max([r[2] or 1 for r in res])
    desc = (f"{a.steps} full hybrid steps (projection + CFL + {a.n_sub} saturation steps + {a.adam_iters} "
            f"Adam iterations, nothing extrapolated) of mix members 0..{a.steps - 1} (sizes "
            f"{[jobs[k][0].n for k in range(a.steps)]}), run by {workers} spawned single-threaded "
            f"worker processes; value = steps / wall time of the pool; {len(warm)} untimed warm-up steps "
            f"(32^2, 1 Adam iteration) first")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * wall / a.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": workload_config(a, world, [s.n for s in mix]),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle", "sample": desc,
                            "blas_threads_per_process": threads,
                            "single_thread_seconds_per_step": sum(r[0] + r[1] * a.adam_iters for r in res) / len(res)},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def scn_small(count):
    from paper_2604_20731_gb300 import scenario as scn
    return [scn.make_scenario(2, 32, seed=1000 + i) for i in range(count)]


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
def serving_mix(count, seed=3):
    """Config-4 style scenario mix: sizes from {128, 256, 512}, permeability
    contrast sigma ~ U[0.5, 2], injection rate ~ U[0.5, 2], one K seed each."""
    from paper_2604_20731_gb300 import scenario as scn
    import numpy as np
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.choice([128, 256, 512]))
        sigma = float(rng.uniform(0.5, 2.0))
        rate = float(rng.uniform(0.5, 2.0))
        out.append(scn.make_scenario(2, n, seed=1000 + i + 100000 * (seed - 3), sigma=sigma, rate=rate))
    return out


def stream_assignment(sizes, nstreams, policy="lpt"):
    """The stream each resident scenario steps on.  "rr": round robin in mix
    order.  "lpt": longest processing time first -- scenarios in decreasing
    order of their estimated step work (128-point tiles of the network plus a
    fixed share for the small kernels) each go to the stream with the least
    work so far, so that the streams finish a round together."""
    if policy == "rr":
        return [i % nstreams for i in range(len(sizes))]
    cost = [((n - 1) ** 2 + 127) // 128 + 100 for n in sizes]
    load = [0] * nstreams
    out = [0] * len(sizes)
    for i in sorted(range(len(sizes)), key=lambda i: (-cost[i], i)):
        k = min(range(nstreams), key=lambda k: (load[k], k))
        out[i] = k
        load[k] += cost[i]
    return out


def batches_by_stream(items, on, groups):
    """The batched form's batches: the scenarios on stream k form batch
    k mod groups, so that the scenarios sharing a stream share a batch (a
    stream holding members of two batches would hold one batch's saturation
    work behind the other's training).  groups <= 0: no batches."""
    if groups <= 0:
        return []
    out = [[x for i, x in enumerate(items) if on[i] % groups == g] for g in range(groups)]
    return [b for b in out if b]


def plain_method_c1(a, scn, HybridSolver, device):
    """Configuration 1: the plain method of Sec. 7 on 32 x 32 elements in FP64.
    Each step is the Galerkin pressure, solved directly on the GPU, followed by
    n_sub explicit saturation steps with the CFL step size.  Timed with CUDA
    events on the solver's stream.  Reported beside it: the error against the
    oracle's plain step and the oracle's own time on the host cores."""
    import numpy as np
    import torch
    from oracle.hybrid import plain_step
    sc = scn.make_scenario(2, 32, seed=1000)
    st = torch.cuda.Stream(device=device)
    s = HybridSolver(sc, width=None, ads_dtype="f64", stream=st)
    s.plain_step(a.n_sub)
    t0 = time.perf_counter()
    S_ref, P_ref, dt_ref = plain_step(sc, sc.S0_or_zero(), a.n_sub, cfl=0.1)
    cpu_ms = (time.perf_counter() - t0) * 1e3
    rel = lambda x, y: float(np.abs(x - y).max() / np.abs(y).max())
    err = {"pressure_rel_linf_vs_oracle_direct": rel(s.get("P"), P_ref),
           "saturation_rel_linf_vs_oracle": rel(s.get("S"), S_ref),
           "dt_rel": abs(float(s.get("DT")[0]) - dt_ref) / dt_ref}
    for _ in range(3):
        s.plain_step(a.n_sub)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(a.c1_steps):
        s.plain_step(a.n_sub)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.c1_steps
    e0.record(st)
    for _ in range(a.c1_steps):
        s.galerkin_pressure()
    e1.record(st)
    torch.cuda.synchronize()
    ms_gal = e0.elapsed_time(e1) / a.c1_steps
    s.get("S")  # a bounded wait that gave up, or a non-finite pivot, fails here
    s.close()
    n = 32
    nu, bw = n * n, 2 * n + 2
    return {"steps_per_s": 1e3 / ms, "ms_per_step": ms, "galerkin_pressure_ms": ms_gal,
            "cholesky_flop": nu * bw * (bw + 1), "error": err,
            "oracle_ms_per_step": cpu_ms, "oracle_cores": 1,
            "note": f"32^2 elements, FP64, {a.n_sub} saturation steps per step, CFL dt; the Galerkin "
                    "pressure (assembly + banded Cholesky + two triangular sweeps, one thread block "
                    "for the sequential pivots) is latency-bound; the oracle uses SuperLU"}


def large_configs(a, scn, HybridSolver, device):
    """Configurations 3 (2D, 1024^2 elements) and 5 (3D, 128^3 elements, K_z =
    0.1 K), one scenario each in mixed precision: FP32 saturation with FP64
    factors and the 128-wide network with BF16 tensor-core products (FP32
    accumulation).  Reports the per-kernel Adam-iteration and saturation
    sub-step times (CUDA events inside the library) and the hybrid step
    (CUDA events on the solver's stream, after one warm-up step); configuration
    5 also with 8 activation-recomputation chunks."""
    import torch
    out = {}
    hp = HybridSolver.hybrid_params(n_sub=a.n_sub, adam_iters=a.adam_iters, lr=a.lr)
    cases = (("c3_2d_1024_w128", 2, 1024, 0), ("c5_3d_128_w128", 3, 128, 0),
             ("c5_3d_128_w128_recompute8", 3, 128, 8))
    for name, dim, n, chunks in cases:
        sc = scn.make_scenario(dim, n, seed=1000, kz_ratio=0.1 if dim == 3 else 1.0)
        st = torch.cuda.Stream(device=device)
        s = HybridSolver(sc, width=128, crv_dtype="bf16", ads_dtype="f32", stream=st, act_chunks=chunks)
        s.set_theta(scn.make_theta0(dim, 128, 4, seed=7))
        s.update_coefficients()
        s.pretrain(5, a.lr)
        prof = s.profile_train(5)
        sat = s.profile_saturation(5)
        s.hybrid_step(hp, stats=False)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(a.large_steps):
            s.hybrid_step(hp, stats=False)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / a.large_steps
        s.get("S")  # a bounded wait that gave up fails here
        s.close()
        it_ms = sum(prof.values())
        npts = (n - 1) ** dim
        out[name] = {"hybrid_step_ms": ms, "adam_iteration_ms": it_ms,
                     "point_iterations_per_s": npts / (it_ms * 1e-3), "kernel_ms": prof,
                     "saturation_substep_ms": sum(sat.values()), "saturation_kernel_ms": sat,
                     "act_chunks": chunks, "hybrid_steps_timed": a.large_steps}
    return out


QUAD_FLOP_PER_ELEMENT = 600      # sum-factorised quadrature of one element (3 x 3 Gauss points)
QUAD_FP32_OPS_PER_ELEMENT = 513  # FP32 pipe operations of k_quad_xsweep_2d per element, counted in its source


def unit_rates():
    """Measured per-SM-per-clock rates of the special-function unit and the
    FP32 pipe (ads_measure_unit_rates), or None if the probe failed."""
    import ctypes as C
    from paper_2604_20731_gb300 import _lib
    lib = _lib.load()
    out = (C.c_double * 11)()
    if lib.ads_measure_unit_rates(out, 11) != 0:
        return None
    names = ["ex2", "rcp", "tanh_pair", "ffma", "ffma2"]
    return {"per_sm_per_clock": {k: out[5 + i] for i, k in enumerate(names)},
            "per_s_at_probe_clock": {k: out[i] for i, k in enumerate(names)},
            "probe_sm_mhz": out[10]}


# FP64 work of the degree-p element kernel per element, counted from its
# loops: per Gauss point S, dP/dx, dP/dy (3 Q^2 + 3 Q FMA), the integrand
# (~40 operations with the sources) and the (p+1)^2 test-function updates
# (4 Q^2); two flops per FMA.  Q = p + 1 points per axis.
def degree_flop_per_element(p):
    q = p + 1
    return q * q * 2 * (7 * q * q + 3 * q + 40)


def degree_step_bench(n, scn, steps=10):
    """The saturation step for B-splines of degree 2, 3 and 4 (FP64, the
    generic path, ads_degree_step) on an n^2 mesh: ms per step by CUDA events
    over `steps` steps after two untimed ones, element-steps/s, and the
    element kernel's FP64 rate against the FP64 peak (2 FMA per clock per SM
    on this GPU: 152 x 2 x 2 x 2070 MHz = 1.26 TFLOP/s)."""
    import ctypes as C
    import numpy as np
    import torch
    from paper_2604_20731_gb300 import _lib
    from paper_2604_20731_gb300.solver import make_params
    lib = _lib.load()
    dev = torch.device("cuda", 0)
    out = {"mesh": f"{n}^2 elements", "fp64_peak_tflops": 152 * 2 * 2 * SM_MAX_MHZ * 1e6 / 1e12}
    for p in (2, 3, 4):
        sc = scn.make_scenario(2, n, seed=1000, S0="random")
        params = make_params(sc, "f64")
        plan = C.c_void_p()
        if lib.ads_degree_plan_create(C.byref(params), p, C.byref(plan)) != 0:
            out[f"p{p}"] = None
            continue
        nb = n + p
        rng = np.random.default_rng(p)
        K = torch.from_numpy(np.ascontiguousarray(sc.K, dtype=np.float64)).to(dev)
        S = torch.from_numpy(rng.uniform(0, 1, size=(nb, nb))).to(dev)
        P = torch.from_numpy(rng.normal(size=(nb, nb))).to(dev)
        o1, o2 = torch.empty_like(S), torch.empty_like(S)
        st = torch.cuda.Stream(device=dev)
        h = C.c_void_p(st.cuda_stream)
        torch.cuda.synchronize()
        for _ in range(2):
            lib.ads_degree_step(plan, K.data_ptr(), None, S.data_ptr(), P.data_ptr(), 1e-4, o1.data_ptr(), h)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        src, dst = o1, o2
        for _ in range(steps):
            rc = lib.ads_degree_step(plan, K.data_ptr(), None, src.data_ptr(), P.data_ptr(), 1e-4,
                                     dst.data_ptr(), h)
            src, dst = dst, src
        e1.record(st)
        st.synchronize()
        lib.ads_degree_plan_destroy(plan)
        ms = e0.elapsed_time(e1) / steps
        fl = degree_flop_per_element(p) * n * n
        out[f"p{p}"] = {"ms_per_step": ms, "element_steps_per_s": n * n / (ms / 1e3), "status": rc,
                        "flop_per_element": degree_flop_per_element(p),
                        "fp64_tflops_whole_step": fl / (ms / 1e3) / 1e12,
                        "frac_of_fp64_peak": fl / (ms / 1e3) / 1e12 / out["fp64_peak_tflops"]}
    return out


def saturation_roofline(n, scn, HybridSolver, rates=None):
    """One 2D saturation sub-step (quadrature + x sweep, y sweep, mass
    bookkeeping) on an n^2 mesh, FP32 and FP64, timed per kernel with CUDA
    events (20 sub-steps after 2 untimed).  Algorithmic bytes: the quadrature
    reads S, P (n+2)^2 and K (n+1)^2 and writes the x-swept rows and the rows
    strips share (Xm, Xs); the y sweep reads Xm and Xs and writes S.  Each
    sub-step's arrays total > L2 at n = 4096."""
    import numpy as np
    peaks, kind = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    sc = scn.make_scenario(2, n, seed=1000, S0="random")
    x = np.linspace(0.0, 1.0, n + 2)
    P = np.outer(np.sin(np.pi * x), np.cos(2 * np.pi * x)) * 10.0
    out = {"mesh": f"{n}^2 elements", "hbm_peak_gbs": hbm, "peak_note": kind}
    for dt, es in (("f32", 4), ("f64", 8)):
        s = HybridSolver(sc, width=None, ads_dtype=dt)
        s.set_pressure(P)
        s.saturation_step(1e-6, 2)
        ms = s.profile_saturation(20)
        s.close()
        nb = n + 2
        re = 4 if 6 * nb * es <= 110 * 1024 else 2
        csz = {4: 2, 2: 4}[re]  # strips per quadrature cluster: one spill pair per cluster
        nsp = 2 * (((n + re - 1) // re + csz - 1) // csz - 1)
        quad_b = es * (2 * nb * nb + (n + 1) ** 2 + nb * nb + nsp * nb)
        ysw_b = es * (2 * nb * nb + nsp * nb)
        tot = sum(ms.values())
        # the line sweep's algorithmic traffic: one read and one write of
        # every DOF per axis (the x sweep's share is fused into the quadrature)
        ysw_alg = 2 * es * nb * nb
        out[dt] = {"ms_per_substep": tot, "kernel_ms": ms,
                   "element_steps_per_s": n * n / (tot * 1e-3),
                   "quad_xsweep_gbs": quad_b / (ms["quad_xsweep"] * 1e-3) / 1e9,
                   "ysweep_gbs_algorithmic": ysw_alg / (ms["ysweep"] * 1e-3) / 1e9,
                   "ysweep_frac_of_hbm": ysw_alg / (ms["ysweep"] * 1e-3) / 1e9 / hbm,
                   "ysweep_gbs_moved": ysw_b / (ms["ysweep"] * 1e-3) / 1e9,
                   "ysweep_frac_of_hbm_moved": ysw_b / (ms["ysweep"] * 1e-3) / 1e9 / hbm,
                   "quad_xsweep_frac_of_hbm": quad_b / (ms["quad_xsweep"] * 1e-3) / 1e9 / hbm,
                   "bytes_per_substep": {"quad_xsweep_moved": quad_b, "ysweep_algorithmic": ysw_alg,
                                         "ysweep_moved": ysw_b}}
        if dt == "f32" and rates:
            ffma = rates["per_sm_per_clock"]["ffma"]
            peak_flop = 2.0 * ffma * N_SM * SM_MAX_MHZ * 1e6
            peak_ops = ffma * N_SM * SM_MAX_MHZ * 1e6
            tq = ms["quad_xsweep"] * 1e-3
            out[dt]["quad_alu"] = {
                "bound": "alu", "unit": "TFLOP/s",
                "achieved": QUAD_FLOP_PER_ELEMENT * n * n / tq / 1e12, "peak": peak_flop / 1e12,
                "frac": QUAD_FLOP_PER_ELEMENT * n * n / tq / peak_flop,
                "flop_per_element": QUAD_FLOP_PER_ELEMENT,
                "fp32_ops_per_element": QUAD_FP32_OPS_PER_ELEMENT,
                "fp32_issue_frac": QUAD_FP32_OPS_PER_ELEMENT * n * n / tq / peak_ops,
                "peak_note": f"measured FP32 fma rate {ffma:.1f} results/clock/SM x {N_SM} SMs x "
                             f"{SM_MAX_MHZ:.0f} MHz x 2 flop"}
    out["note"] = ("the quadrature + x sweep is bound by FP32 (FP64) instruction issue, not by "
                   "HBM; the y sweep is the bandwidth-bound line solve")
    return out


def summary_line(value, plain, err, sat, roof, e2e):
    """The few numbers the line is about, short enough to survive truncation."""
    out = {"steps_per_s": round(value, 2)}
    if plain:
        out["mp_batched_over_plain_fp64"] = round(plain["mp_batched_over_plain_fp64"], 1)
    if err:
        ms = err["mix_pressure_summary"]
        out["mix_pressure_rel_l2_median_max"] = [round(ms["median"], 4), round(ms["max"], 4)]
        out["mix_pressure_at_or_below_1e-2"] = f"{ms['at_or_below_1e-2']}/{ms['sampled']}"
        out["mix_saturation_rel_linf_max"] = max(x["rel_linf"] for x in err["mix_saturation_rel_linf_one_fp32_step"])
    if roof and roof.get("frac") is not None:
        out["roofline"] = f"{roof['kernel']} {roof['frac']:.3f} of measured {roof['unit']}"
    if sat and sat.get("f32"):
        f = sat["f32"]
        out["ysweep_frac_of_hbm"] = round(f["ysweep_frac_of_hbm"], 3)
        if f.get("quad_alu"):
            out["quad_fp32_frac"] = round(f["quad_alu"]["frac"], 3)
    if e2e:
        out["e2e_steps_per_s"] = round(e2e["value"], 2)
    return out


def base_network(a, scn, HybridSolver, theta0):
    """The base network the scenarios start from: the homogeneous 256^2
    scenario (K = 1, rate 1, the wells of the mix) trained from the Xavier
    network, half the iterations at lr 1e-3 and half at 3e-4.  Returns the
    parameters (or None with base_iters 0) and its error record."""
    import numpy as np
    if a.base_iters <= 0:
        return None, None
    from oracle.crvpinn import CrvOracle
    sc = scn.make_scenario(2, 256, seed=1000, sigma=0.0, rate=1.0)
    t0 = time.perf_counter()
    s = HybridSolver(sc, width=a.width, crv_dtype="bf16", ads_dtype="f32")
    s.set_theta(theta0)
    s.pretrain(a.base_iters // 2, 1e-3)
    s.pressure_update(a.base_iters - a.base_iters // 2, 3e-4)
    th = s.get("THETA").astype(np.float64)
    sec = time.perf_counter() - t0
    crv = CrvOracle(sc)
    alpha, f = crv.coefficients(sc.S0_or_zero())
    ustar = crv.direct_solution(alpha, f)
    s.project_pressure()
    e = float(np.linalg.norm(s.get("U") - ustar) / np.linalg.norm(ustar))
    s.close()
    return th, {"scenario": "256^2, K = 1, rate 1", "iterations": a.base_iters, "seconds": sec,
                "pressure_rel_l2": e}


def stated_error(a, mix, sizes, ctxs, hp, theta0, scn, HybridSolver):
    """The error the throughput is measured at (see run_ours)."""
    import numpy as np
    from oracle.ads import AdsOracle
    from oracle.crvpinn import CrvOracle
    members, sat = [], []
    for n in sorted(set(sizes)):
        idx = [i for i, m in enumerate(mix) if m.n == n]
        sig = [float(np.log(mix[i].K).std()) for i in idx]
        order = np.argsort(sig)
        picks = sorted({int(order[0]), int(order[len(order) // 2]), int(order[-1])})
        for k in picks:
            j = idx[k]
            s, sc = ctxs[j], mix[j]
            S_now = s.get("S")
            crv = CrvOracle(sc)
            alpha, f = crv.coefficients(S_now)
            ustar = crv.direct_solution(alpha, f)
            s.project_pressure()
            e = float(np.linalg.norm(s.get("U") - ustar) / np.linalg.norm(ustar))
            members.append({"member": j, "n": n, "log_k_std": round(sig[k], 3),
                            "rate": round(sc.sources[0].rate, 3), "pressure_rel_l2": e})
        j = idx[int(order[len(order) // 2])]
        s, sc = ctxs[j], mix[j]
        S_now, P_now = s.get("S"), s.get("P")
        dt_now = float(s.get("DT")[0])
        s2 = HybridSolver(sc, width=None, ads_dtype="f32")
        s2.set_saturation(S_now)
        s2.set_pressure(P_now)
        s2.saturation_step(dt_now, 1)
        ref = AdsOracle(sc).step(S_now, P_now, dt_now)
        sat.append({"member": j, "n": n,
                    "rel_linf": float(np.abs(s2.get("S") - ref).max() / max(np.abs(ref).max(), 1e-300))})
        s2.close()
    pe = [m["pressure_rel_l2"] for m in members]

    def pressure_error(scen, dtn, steps):
        crv = CrvOracle(scen)
        sa = HybridSolver(scen, width=a.width, crv_dtype=dtn, ads_dtype="f32")
        sa.set_theta(theta0)
        sa.pretrain(a.err_iters, 1e-3)

        def rel():
            alpha, f = crv.coefficients(sa.get("S"))
            ustar = crv.direct_solution(alpha, f)
            sa.project_pressure()
            return float(np.linalg.norm(sa.get("U") - ustar) / np.linalg.norm(ustar))

        out = [rel()]
        for _ in range(steps):
            sa.hybrid_step(hp)
            out.append(rel())
        sa.close()
        return out

    c2 = scn.make_scenario(2, 256, seed=1000)
    p_c2 = {dtn: pressure_error(c2, dtn, a.err_steps) for dtn in ("bf16", "f32")}
    return {
        "mix_pressure_rel_l2": members,
        "mix_pressure_summary": {"sampled": len(pe), "median": float(np.median(pe)), "max": float(max(pe)),
                                 "at_or_below_1e-2": int(sum(x <= 1e-2 for x in pe))},
        "mix_pressure_note": (f"members of the timed mix after {a.pretrain} admission iterations, "
                              f"{max(a.warmup, 3)} warm-up and {a.steps} timed hybrid steps of {a.adam_iters} "
                              "iterations; network at its current parameters vs the direct discrete solution "
                              "for the member's current saturation"),
        "mix_saturation_rel_linf_one_fp32_step": sat,
        "c2_pressure_scenario": "256^2, sigma 1, correlation length 0.1, seed 1000",
        "c2_pressure_rel_l2_bf16": p_c2["bf16"][0], "c2_pressure_rel_l2_fp32": p_c2["f32"][0],
        "c2_pressure_rel_l2_after_each_hybrid_step_bf16": p_c2["bf16"][1:],
        "c2_pressure_rel_l2_after_each_hybrid_step_fp32": p_c2["f32"][1:],
        "c2_note": f"{a.err_iters} Adam iterations (lr 1e-3) from the Xavier network, then {a.err_steps} hybrid steps",
    }


def run_ours(a, world, rank, local):
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    import __graft_entry__ as g
    if rank == 0:
        g.build()
    barrier(world)
    from paper_2604_20731_gb300 import scenario as scn
    from paper_2604_20731_gb300.solver import HybridSolver, Server, hybrid_step_batch, hybrid_step_batch_profile

    rates = unit_rates() if rank == 0 else None
    if a.only_saturation:
        if rank == 0:
            print(json.dumps({"saturation": saturation_roofline(a.sat_n, scn, HybridSolver, rates)}), flush=True)
        return 0
    if a.only_degree:
        if rank == 0:
            print(json.dumps({"degree_p": degree_step_bench(a.degree_n, scn)}), flush=True)
        return 0
    hp = HybridSolver.hybrid_params(n_sub=a.n_sub, dt=1.0, dt_policy=1, cfl=0.1, src_frac=0.05,
                                    adam_iters=a.adam_iters, lr=a.lr)
    theta0 = scn.make_theta0(2, a.width, 4, seed=7)
    mix = serving_mix(a.scenarios, seed=3 + rank)
    sizes = [sc.n for sc in mix]
    # warm start: every scenario's network starts from one base network,
    # trained once (outside every timed region) on the homogeneous scenario
    # K = 1, rate 1, with its output layer scaled by the scenario's rate
    base, base_info = base_network(a, scn, HybridSolver, theta0)

    def theta_start(sc):
        if base is None:
            return theta0
        th = base.copy()
        th[-(a.width + 1):] *= sc.sources[0].rate  # output layer W_5, b_5
        return th

    # ---- (1) batched mixed precision, scenarios resident: the headline ----
    streams = [torch.cuda.Stream(device=device) for _ in range(a.streams)]
    on = stream_assignment(sizes, a.streams, a.assign)
    ctxs = []
    for i, sc in enumerate(mix):
        s = HybridSolver(sc, width=a.width, crv_dtype="bf16", ads_dtype="f32", stream=streams[on[i]])
        s.set_concurrency(min(a.streams, len(mix)))
        s.set_theta(theta_start(sc))
        ctxs.append(s)
    # admission training of every resident scenario, side by side on the streams
    t_adm = time.perf_counter()
    if a.pretrain > 0:
        for s in ctxs:
            s.pretrain(a.pretrain, a.lr, sync=False)
    torch.cuda.synchronize()
    admission_s = time.perf_counter() - t_adm
    batches = batches_by_stream(ctxs, on, a.groups)

    def step_all():
        if batches:
            for b in batches:
                hybrid_step_batch(b, hp)
        else:
            for s in ctxs:
                s.hybrid_step(hp, stats=False)

    for _ in range(max(a.warmup, 3)):
        step_all()
    torch.cuda.synchronize()
    # raw samples to a CSV when ADSGB_CLOCKS_CSV names a file (rank appended)
    csv_path = os.environ.get("ADSGB_CLOCKS_CSV")
    clocks = ClockSampler(local, path=f"{csv_path}.rank{rank}" if csv_path else None)
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in streams]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in streams]
    round_ev = [[torch.cuda.Event(enable_timing=True) for _ in streams] for _ in range(a.steps)]
    barrier(world)
    torch.cuda.synchronize()
    l0 = sum(s.kernel_launches() for s in ctxs)
    clocks.start()
    time.sleep(0.3)
    for k, st in enumerate(streams):
        ev0[k].record(st)
    for r in range(a.steps):
        step_all()
        for k, st in enumerate(streams):
            round_ev[r][k].record(st)
    for k, st in enumerate(streams):
        ev1[k].record(st)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = sum(s.kernel_launches() for s in ctxs) - l0
    # every kernel's bounded waits completed (a timed-out wait leaves a status
    # bit that ads_get reports)
    for s in ctxs:
        s.get("DT")
    total_ms = max(ev0[0].elapsed_time(e) for e in ev1)
    round_end = [max(ev0[0].elapsed_time(e) for e in round_ev[r]) for r in range(a.steps)]
    round_ms = [round_end[0]] + [round_end[r] - round_end[r - 1] for r in range(1, a.steps)]
    total_ms = max_over_ranks(total_ms, world, device)
    steps_done = a.steps * len(ctxs) * world
    value = steps_done / (total_ms / 1e3)

    # ---- stated error of the measured mix (rank 0, after the timed rounds) ----
    #  * pressure: for each mesh size, the members of the mix with the lowest,
    #    median and highest log-K spread, in the state the timed rounds left
    #    them: relative L2 of the network pressure (current parameters) against
    #    the direct discrete solution for the member's current saturation;
    #  * saturation: one FP32 sub-step from the GPU state of one member per
    #    size against the FP64 oracle (relative L-inf);
    #  * the single-scenario study of configuration 2 (256^2, sigma 1): the
    #    network trained for `err_iters` iterations, then `err_steps` hybrid
    #    steps, BF16 and FP32 networks side by side.
    err = None
    if rank == 0 and not a.no_error:
        err = stated_error(a, mix, sizes, ctxs, hp, theta0, scn, HybridSolver)

    # ---- roofline of the dominant kernel (live CUDA events) ----
    # With batches, the timed region runs grouped launches: one grouped
    # iteration of the first batch, replayed with events between its kernels,
    # gives their times in the shape the timed region runs them.
    grouped = None
    if batches and rank == 0:
        grouped = {"members": len(batches[0]),
                   "points": sum((s.sc.n - 1) ** 2 for s in batches[0]),
                   "ms": hybrid_step_batch_profile(batches[0], a.profile_iters)}
    # (and each size's kernels in their full-GPU launch shape: one context alone)
    prof_by_n = {}
    for n in sorted(set(sizes)):
        j = sizes.index(n)
        ctxs[j].set_concurrency(1)
        prof_by_n[n] = ctxs[j].profile_train(a.profile_iters)
    count = {n: sizes.count(n) for n in prof_by_n}
    tot = {}
    for n, pr in prof_by_n.items():
        for k, v in pr.items():
            tot[k] = tot.get(k, 0.0) + v * count[n]
    dom = max(tot, key=tot.get)
    peaks, peak_kind = measured_peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    fwd_f, bwd_f = mlp_flops_per_point(2, a.width)
    flops_pt = {"mlp_fwd": fwd_f, "mlp_bwd": bwd_f}
    nbig = max(prof_by_n)
    roof = {"kernel": dom, "share_of_mix_kernel_time": tot[dom] / sum(tot.values())}
    if dom == "mlp_fwd" and rates:
        # the forward's binding unit is the special-function pipe: each of
        # the 4 hidden layers' W units of a point takes one tanh = one ex2 +
        # one rcp; the peak is the measured rate of that pair
        M = (nbig - 1) ** 2
        t = prof_by_n[nbig][dom] * 1e-3
        ops = 4 * a.width * M
        ach = ops / t / 1e12
        pair = rates["per_sm_per_clock"]["tanh_pair"]
        pk = N_SM * pair * sm_mhz * 1e6 / 1e12
        fl = flops_pt[dom] * M
        tpk = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1700.0)))
        tr = traffic_record(dom + "_tc")
        roof.update({"bound": "alu", "achieved": ach, "peak": pk, "unit": "T tanh/s",
                     "frac": ach / pk, "traffic": tr["bytes_per_launch"] if tr else None,
                     "peak_note": f"measured ex2 + rcp pair rate {pair:.2f}/clock/SM (ex2 "
                                  f"{rates['per_sm_per_clock']['ex2']:.1f}, rcp {rates['per_sm_per_clock']['rcp']:.1f}) "
                                  f"x {N_SM} SMs x {sm_mhz:.0f} MHz",
                     "algorithmic_ops_per_launch": ops, "avg_launch_ms": prof_by_n[nbig][dom],
                     "tensor_achieved_tflops": fl / t / 1e12, "tensor_frac_of_sustained_bf16": fl / t / 1e12 / tpk,
                     "workload": f"{nbig}^2 member of the mix"})
    elif dom in flops_pt:
        M = (nbig - 1) ** 2
        fl = flops_pt[dom] * M
        ach = fl / (prof_by_n[nbig][dom] * 1e-3) / 1e12
        pk = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1700.0)))
        tr = traffic_record(dom + "_tc")
        roof.update({"bound": "tensor", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                     "frac": ach / pk, "traffic": tr["bytes_per_launch"] if tr else None,
                     "peak_note": f"BF16 dense, sustained, {peak_kind}",
                     "algorithmic_flop_per_launch": fl, "avg_launch_ms": prof_by_n[nbig][dom],
                     "workload": f"{nbig}^2 member of the mix"})
    elif dom in ("dst_gemm", "idst_gemm_loss"):
        m = nbig - 1
        fl = 2.0 * m ** 3
        ach = fl / (prof_by_n[nbig][dom] * 1e-3) / 1e12
        pk = N_SM * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
        tr = traffic_record(dom)
        roof.update({"bound": "alu", "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
                     "traffic": tr["bytes_per_launch"] if tr else None,
                     "peak_note": f"FP32 FFMA: {N_SM} SMs x {FP32_LANES_PER_SM} lanes x 2 x {sm_mhz:.0f} MHz",
                     "algorithmic_flop_per_launch": fl, "avg_launch_ms": prof_by_n[nbig][dom],
                     "workload": f"{nbig}^2 member of the mix"})
    else:
        roof.update({"bound": "latency", "achieved": None, "peak": None, "unit": None, "frac": None,
                     "traffic": None})
    if grouped:
        # the timed region's own kernels: the dominant grouped kernel of the
        # first batch, per launch (all of the batch's points)
        gms = grouped["ms"]
        gdom = max(gms, key=gms.get)
        P = grouped["points"]
        per_ctx = roof
        roof = {"kernel": gdom + " (grouped)", "share_of_batch_iteration": gms[gdom] / sum(gms.values()),
                "workload": f"one grouped launch over batch 0: {grouped['members']} scenarios, {P} points",
                "avg_launch_ms": gms[gdom], "per_scenario_launch_shape": per_ctx}
        tr = traffic_record(gdom + "_tc_grp")
        traffic = tr["bytes_per_point"] * P if tr and "bytes_per_point" in tr else None
        t = gms[gdom] * 1e-3
        if gdom in flops_pt:
            fl = flops_pt[gdom] * P
            tpk = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1700.0)))
            if gdom == "mlp_fwd" and rates:
                ops = 4 * a.width * P
                pair = rates["per_sm_per_clock"]["tanh_pair"]
                pk = N_SM * pair * sm_mhz * 1e6 / 1e12
                roof.update({"bound": "alu", "achieved": ops / t / 1e12, "peak": pk, "unit": "T tanh/s",
                             "frac": ops / t / 1e12 / pk, "traffic": traffic,
                             "peak_note": f"measured ex2 + rcp pair rate {pair:.2f}/clock/SM x {N_SM} SMs x "
                                          f"{sm_mhz:.0f} MHz",
                             "algorithmic_ops_per_launch": ops, "tensor_achieved_tflops": fl / t / 1e12,
                             "tensor_frac_of_sustained_bf16": fl / t / 1e12 / tpk})
            else:
                roof.update({"bound": "tensor", "achieved": fl / t / 1e12, "peak": tpk, "unit": "TFLOP/s",
                             "frac": fl / t / 1e12 / tpk, "traffic": traffic,
                             "peak_note": f"BF16 dense, sustained, {peak_kind}",
                             "algorithmic_flop_per_launch": fl})
        else:
            roof.update({"bound": "latency", "achieved": None, "peak": None, "unit": None, "frac": None,
                         "traffic": None})
        if traffic is not None:
            roof["traffic_note"] = (f"{tr['bytes_per_point']:.1f} B per point from a smaller grouped capture "
                                    f"(profiles/traffic.txt), times the launch's {P} points")
    for s in ctxs:
        s.close()
    del ctxs

    # ---- (2) end to end: the same mix through the C-ABI server ----
    e2e = None
    server_stats = None
    if a.e2e_steps > 0:
        srv = Server(hbm_budget=int(a.budget_gb * (1 << 30)), max_active=len(mix), n_streams=a.streams)
        rng = np.random.default_rng(3 + rank)
        arrivals = np.cumsum(rng.exponential(a.arrival_ms / 1e3, size=len(mix)))
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        ids = []
        for i, sc in enumerate(mix):
            wait = t0 + arrivals[i] - time.perf_counter()
            if wait > 0:
                time.sleep(wait)
            ids.append(srv.submit(sc, n_steps=a.e2e_steps, hp=hp, width=a.width, crv_dtype="bf16",
                                  ads_dtype="f32", pretrain_iters=a.pretrain, pretrain_lr=a.lr,
                                  theta0=theta_start(sc)))
        for rid in ids:
            srv.wait(rid, timeout_s=900)
        torch.cuda.synchronize()
        el = max_over_ranks(time.perf_counter() - t0, world, device)
        server_stats = srv.stats()
        srv.close()
        nb_bytes = sum(((sc.n + 2) ** 2) for sc in mix) * 8
        nn_bytes = sum(((sc.n + 1) ** 2) for sc in mix) * 8
        e2e = {"value": len(mix) * a.e2e_steps * world / el, "unit": UNIT,
               "h2d_bytes_per_step": (nn_bytes + nb_bytes) / (len(mix) * a.e2e_steps),
               "d2h_bytes_per_step": 2 * nb_bytes / (len(mix) * a.e2e_steps),
               "steps_per_scenario": a.e2e_steps, "arrivals": f"Poisson, mean {a.arrival_ms} ms",
               "budget_gb": a.budget_gb, "pretrain_at_admission": a.pretrain,
               "start": "base network" if base is not None else "Xavier",
               "p50_step_ms": server_stats["p50_step_ms"], "p99_step_ms": server_stats["p99_step_ms"],
               "peak_resident": server_stats["peak_active"]}

    # ---- (3) plain FP64, one scenario at a time, on a sample of the mix ----
    plain = None
    if rank == 0 and a.plain_steps > 0:
        per_n = {}
        for n in sorted(set(sizes)):
            sc = scn.make_scenario(2, n, seed=1000)
            s = HybridSolver(sc, width=a.width, crv_dtype="f64", ads_dtype="f64")
            s.set_theta(theta0)
            s.hybrid_step(hp, stats=False)
            s.sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(a.plain_steps):
                s.hybrid_step(hp, stats=False)
            s.sync()
            per_n[n] = (time.perf_counter() - t0) * 1e3 / a.plain_steps
            s.close()
        mean_ms = sum(per_n[n] for n in sizes) / len(sizes)
        plain = {"steps_per_s": 1e3 / mean_ms, "ms_per_step_by_n": per_n,
                 "sample": f"{a.plain_steps} timed FP64 hybrid steps per size (after one warm-up), "
                           "weighted by the mix; FP64 saturation + FP64 CUDA-core network",
                 "mp_batched_over_plain_fp64": value / world / (1e3 / mean_ms)}

    # ---- (4) config 2 as specified: 256^2, FP64 saturation, FP32 network ----
    c2 = None
    if rank == 0 and a.c2_steps > 0:
        sc = scn.make_scenario(2, 256, seed=1000)
        st = torch.cuda.Stream(device=device)
        s = HybridSolver(sc, width=a.width, crv_dtype="f32", ads_dtype="f64", stream=st)
        s.set_theta(theta0)
        s.pretrain(a.pretrain, a.lr)
        for _ in range(3):
            s.hybrid_step(hp, stats=False)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(a.c2_steps):
            s.hybrid_step(hp, stats=False)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / a.c2_steps
        c2 = {"steps_per_s": 1e3 / ms, "ms_per_step": ms, "kernel_ms": s.profile_train(a.profile_iters),
              "note": "single scenario, L2-resident working set"}
        s.close()

    # ---- (4b) config 1: the plain method (Galerkin pressure, direct FP64 solve) ----
    c1 = None
    if rank == 0 and a.c1_steps > 0:
        c1 = plain_method_c1(a, scn, HybridSolver, device)

    # ---- (4c) configurations 3 and 5: the 128-wide network in 2D and 3D ----
    large = None
    if rank == 0 and a.large_steps > 0:
        large = large_configs(a, scn, HybridSolver, device)

    # ---- (4d) saturation kernels on a mesh larger than L2 (FP32 and FP64) ----
    sat = None
    if rank == 0 and a.sat_n > 0:
        sat = saturation_roofline(a.sat_n, scn, HybridSolver, rates)
    degree = None
    if rank == 0 and a.degree_n > 0:
        degree = degree_step_bench(a.degree_n, scn)

    # ---- (5) CPU baseline (rank 0, N=1 only): the oracle on the mix ----
    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cpu = oracle_baseline(a, mix, sizes)

    if rank == 0:
        rs = sorted(round_ms)
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
               "warmup": a.warmup, "ms_per_step": total_ms / (a.steps * len(mix)),
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": "bf16+f32", "data": "synthetic (log-normal K GRF, Gaussian wells)",
               "config": workload_config(a, world, sizes),
               "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
               "gpu_launches": launches, "gpu_launches_before_timed": l0, "clocks": clk,
               # details first, the summary a reader looks for last (a truncated
               # record keeps the end of the line)
               "kernel_ms_by_n": prof_by_n, "kernel_ms_grouped": grouped, "unit_rates": rates, "server": server_stats,
               "c3_c5_w128": large, "c2_fp64_sat_fp32_net": c2, "c1_plain_galerkin": c1,
               "saturation": sat, "degree_p": degree, "base_network": base_info,
               "admission_training_s": admission_s,
               "error": err,
               "latency_note": "resident run: a scenario's step latency is the round time (all "
                               "scenarios step once per round); e2e holds the server's per-step latency",
               "plain_fp64": plain,
               "summary": summary_line(value, plain, err, sat, roof, e2e),
               "p50_step_ms": rs[len(rs) // 2],
               "p99_step_ms": rs[min(len(rs) - 1, int(math.ceil(0.99 * len(rs))) - 1)]}
        print(json.dumps(out), flush=True)
    return 0


def main():
    a = args_parse()
    world, rank, local = dist_setup()
    if a.impl == "reference":
        rc = run_reference(a, world, rank)
    else:
        rc = run_ours(a, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
