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


def args_parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--width", type=int, default=64)
    ap.add_argument("--adam-iters", type=int, default=100)
    ap.add_argument("--n-sub", type=int, default=10)
    ap.add_argument("--pretrain", type=int, default=500)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-iters", type=int, default=30)
    return ap.parse_args()


def workload_config(a, world):
    return {
        "workload": f"2D {a.n}x{a.n} p=2 FP64 saturation + CRVPINN 2-{a.width}x4-1 FP32 on "
                    f"{a.n + 1}^2 collocation; {a.n_sub} saturation steps + {a.adam_iters} Adam "
                    f"iterations per hybrid step",
        "n": a.n, "collocation": a.n + 1, "mlp": f"2-{a.width}x4-1", "ads_dtype": "f64",
        "crvpinn_dtype": "f32", "n_sub": a.n_sub, "adam_iters": a.adam_iters, "lr": a.lr,
        "dt_policy": "cfl 0.1", "scenarios_per_gpu": 1, "parallelism": f"replicas x{world}",
        "l2": "flushed between timed steps (256 MB write)",
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
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
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
# CPU oracle sample (the baseline and the reference arm)
# ---------------------------------------------------------------------------
def oracle_step_sample(a, adam_sample):
    """Time the oracle on one hybrid step with `adam_sample` Adam iterations
    measured and the rest extrapolated.  Returns (seconds per hybrid step,
    description)."""
    import numpy as np
    from oracle.crvpinn import Adam
    from oracle.hybrid import HybridOracle
    from paper_2604_20731_gb300 import scenario as scn
    sc = scn.make_scenario(2, a.n, seed=1000)
    h = HybridOracle(sc, width=a.width)
    theta = scn.make_theta0(2, a.width, 4, seed=7)
    opt = Adam(theta.size)
    S = sc.S0_or_zero()
    h.crv.gram_solve_lu(np.zeros(h.crv.M))  # the Gram LU is factorised once (Eq. 28)
    t0 = time.perf_counter()
    P = h.project(theta)
    dt = h.ads.cfl_dt(P, cfl=0.1, dt_cap=1.0)
    for _ in range(a.n_sub):
        S = h.ads.step(S, P, dt)
    t1 = time.perf_counter()
    theta, _ = h.train(theta, opt, S, adam_sample, a.lr)
    t2 = time.perf_counter()
    per_iter = (t2 - t1) / adam_sample
    step_s = (t1 - t0) + per_iter * a.adam_iters
    desc = (f"one hybrid step on {a.n}^2: projection + CFL + {a.n_sub} saturation steps measured, "
            f"{adam_sample} of {a.adam_iters} Adam iterations measured and scaled "
            f"({per_iter * 1e3:.1f} ms/iteration)")
    return step_s, desc


def run_reference(a, world, rank):
    if rank != 0:
        return 0
    cores = os.cpu_count()
    for _ in range(a.warmup if a.warmup < 1 else 1):
        oracle_step_sample(a, 1)
    times = []
    desc = ""
    for _ in range(a.steps):
        s, desc = oracle_step_sample(a, 2)
        times.append(s)
    total = sum(times)
    value = a.steps / total
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * total / a.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": workload_config(a, world),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": desc},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
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
    from paper_2604_20731_gb300.solver import HybridSolver

    sc = scn.make_scenario(2, a.n, seed=1000 + rank)
    stream = torch.cuda.Stream(device=device)
    s = HybridSolver(sc, width=a.width, crv_dtype="f32", ads_dtype="f64", stream=stream)
    s.set_theta(scn.make_theta0(2, a.width, 4, seed=7))
    pre_loss = s.pretrain(a.pretrain, a.lr) if a.pretrain > 0 else float("nan")
    hp = s.hybrid_params(n_sub=a.n_sub, dt=1.0, dt_policy=1, cfl=0.1, src_frac=0.05,
                         adam_iters=a.adam_iters, lr=a.lr)
    for _ in range(max(a.warmup, 3)):
        s.hybrid_step(hp, stats=False)
    s.sync()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=device)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(a.steps)]
    clocks = ClockSampler(local, path=os.path.join(ROOT, "gpurun_out", f"clocks_rank{rank}.csv")
                          if os.path.isdir(os.path.join(ROOT, "gpurun_out")) else None)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    l0 = s.kernel_launches()
    clocks.start()
    time.sleep(0.3)
    with torch.cuda.stream(stream):
        for i in range(a.steps):
            flush.fill_(float(i))  # evict the previous step's working set from L2
            ev[i][0].record(stream)
            s.hybrid_step(hp, stats=False)
            ev[i][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = s.kernel_launches() - l0
    barrier(world)
    step_ms = [e0.elapsed_time(e1) for e0, e1 in ev]
    total_ms = max_over_ranks(sum(step_ms), world, device)
    stats = s.hybrid_step(hp, stats=True)  # one more (untimed) for the reported state
    value = a.steps * world / (total_ms / 1e3)

    # ---- roofline of the dominant kernel (live, CUDA events on our stream) ----
    prof = s.profile_train(a.profile_iters)
    sat = s.profile_saturation(10)
    dom = max(prof, key=prof.get)
    fwd_f, bwd_f = mlp_flops_per_point(2, a.width)
    M = (a.n - 1) ** 2
    flops = {"mlp_fwd": fwd_f * M, "mlp_bwd": bwd_f * M}
    peaks, peak_kind = measured_peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = N_SM * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    roof = None
    if dom in flops:
        ach = flops[dom] / (prof[dom] * 1e-3) / 1e12
        tr = traffic_record(dom)
        roof = {"bound": "alu", "kernel": dom, "achieved": ach, "peak": fp32_peak,
                "unit": "TFLOP/s", "frac": ach / fp32_peak,
                "traffic": tr["bytes_per_launch"] if tr else None,
                "peak_note": f"FP32 FFMA peak = {N_SM} SMs x {FP32_LANES_PER_SM} lanes x 2 x "
                             f"{sm_mhz:.0f} MHz (sm_max_mhz of {peak_kind} peaks file)",
                "algorithmic_flop_per_launch": flops[dom], "avg_launch_ms": prof[dom]}
    else:
        roof = {"bound": "alu", "kernel": dom, "achieved": None, "peak": fp32_peak,
                "unit": "TFLOP/s", "frac": None, "traffic": None}

    # ---- stated error (rank 0): saturation step vs oracle, pressure vs direct ----
    err = None
    if rank == 0:
        from oracle.ads import AdsOracle
        from oracle.crvpinn import CrvOracle
        S_now = s.get("S")
        P_now = s.get("P")
        dt_now = float(s.get("DT")[0])
        s2 = HybridSolver(sc, width=None, ads_dtype="f64")
        s2.set_saturation(S_now)
        s2.set_pressure(P_now)
        s2.saturation_step(dt_now, 1)
        ref = AdsOracle(sc).step(S_now, P_now, dt_now)
        sat_err = float(np.abs(s2.get("S") - ref).max() / max(np.abs(ref).max(), 1e-300))
        s2.close()
        crv = CrvOracle(sc)
        alpha, f = crv.coefficients(S_now)
        ustar = crv.direct_solution(alpha, f)
        s.project_pressure()
        u = s.get("U")
        p_err = float(np.linalg.norm(u - ustar) / np.linalg.norm(ustar))
        err = {"saturation_rel_linf_vs_oracle_one_step": sat_err,
               "pressure_rel_l2_vs_direct": p_err,
               "pressure_note": f"after {a.pretrain} pretrain + {a.warmup + a.steps + 1} x "
                                f"{a.adam_iters} Adam iterations"}

    # ---- end to end through the C ABI with host buffers ----
    e2e = None
    if a.e2e_steps > 0:
        nb = a.n + 2
        host_S = torch.empty((nb, nb), dtype=torch.float64, pin_memory=True).numpy()
        host_S[:] = s.get("S")
        ne = a.e2e_steps
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(ne):
            s.set_saturation(host_S)           # H2D: the step's input state
            s.hybrid_step(hp, stats=True)      # D2H: step size, loss, mass balance
            host_S[:] = s.get("S")             # D2H: the step's result
        torch.cuda.synchronize()
        el = max_over_ranks(time.perf_counter() - t0, world, device)
        e2e = {"value": ne * world / el, "unit": UNIT, "h2d_bytes_per_step": nb * nb * 8,
               "d2h_bytes_per_step": nb * nb * 8 + 4 * 8 + 4}

    # ---- CPU baseline (rank 0, N=1 only) ----
    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        t1, _ = oracle_step_sample(a, 1)
        per_iter_est = max(t1 / max(a.adam_iters, 1), 1e-3)
        sample = int(min(max(10.0 / per_iter_est, 2), a.adam_iters))
        st_s, desc = oracle_step_sample(a, min(sample, 20))
        cpu = {"value": 1.0 / st_s, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": desc}

    if rank == 0:
        step_ms_sorted = sorted(step_ms)
        p50 = step_ms_sorted[len(step_ms) // 2]
        p99 = step_ms_sorted[min(len(step_ms) - 1, int(math.ceil(0.99 * len(step_ms))) - 1)]
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
               "warmup": a.warmup, "ms_per_step": total_ms / a.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32",
               "data": "synthetic (log-normal K GRF, Gaussian wells)",
               "config": workload_config(a, world),
               "p50_step_ms": p50, "p99_step_ms": p99,
               "element_steps_per_s": value * a.n_sub * a.n * a.n,
               "collocation_point_iterations_per_s": value * a.adam_iters * M,
               "error": err, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
               "gpu_launches": launches, "clocks": clk,
               "kernel_ms": {"train": prof, "saturation": sat},
               "last_step": stats, "pretrain_loss": pre_loss}
        print(json.dumps(out), flush=True)
    s.close()
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
