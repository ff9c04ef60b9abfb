#!/usr/bin/env python3
"""AIRPF throughput on one GB300: particle-steps/s on the large nonlinear-growth workload
(m = 65536 islands x M = 256 particles, N = 16.8 M, T = 1000 observations simulated from seed 5,
x_t = x/2 + 25 x / (1 + x^2) + 8 cos(1.2 t) + v, v ~ N(0, 10), y_t = x_t^2 / 20 + w, w ~ N(0, 1),
adaptive interaction tau = 0.3, FP32 particles with FP64 island weights and log Z), the largest
single-GPU configuration of the workloads; further legs: the stochastic-volatility workload
(m = 1024 x M = 256), the all-FP64 paths, an M sweep, batched chains, gradients, PMMH and the
change-point model.

A step is one full AIRPF pass over y_1..y_T (every row of the hot path: propagate, weight,
island log-sum-exp, internal resampling, ENF-controlled island interaction, log Z
accumulation), at the next iteration index of the random streams.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl airpf|reference]

Prints one JSON line (rank 0).  --impl reference times the CPU oracle instead.
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

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "AIRPF particle-steps/s and PMCMC iters/s on 1 GB300 at stated log-\u1e90 error"
UNIT = "particle-steps/s"
WORKLOAD = "ngm_m65536_M256_T1000"
M_ISL, M_PART, T_OBS = 65536, 256, 1000
SV_WORKLOAD = "sv_m1024_M256_T1000"
SV_M_ISL, SV_M_PART = 1024, 256
TAU = 0.3
L2_FLUSH_BYTES = 256 << 20
LANES_PER_SM = 128

# Algorithmic lane operations per particle-step of the FP32-mixed path (a definition,
# counted from the algorithm, not from the compiler).  Two particles share one
# Philox4x32-10 block (10 rounds of two 32x32->64 multiplies, counted as 4 operations, and 4
# xors, 9 key-schedule steps of 2 adds: about 100) and one Box-Muller pair (13); the binary
# search over M = 256 takes 8 levels of 7 (index, swizzle, shared-memory load, compare,
# select).
OPS_COMMON = {"philox_half_block": 50, "box_muller_half_pair": 6.5, "island_max": 4,
              "weight_fixed_point": 5, "integer_prefix_sum": 10, "cdf_and_particle_stores": 2,
              "draw_target": 4, "binary_search_M256": 56, "gather": 4}
OPS_MODEL = {"NGM": {"transition": 8, "log_density": 4}, "SV": {"transition": 3, "log_density": 9}}


def ops_per_particle_step(model: str) -> float:
    return sum(OPS_COMMON.values()) + sum(OPS_MODEL[model].values())


# Figures from the committed ncu captures of the kernels named (set to None when the kernel
# changes, until it is captured again): DRAM read + write per launch, issue-active fraction.
NCU = {
    # traffic null: the kernel changed (the search's top five levels by shuffles) after the
    # counters were taken; they read 95200768 B and 0.763 issue active on the build before
    "ngm_island_step": {"dram_bytes_per_launch": None, "issue_active": 0.763,
                        "source": "ncu smsp__issue_active of airpf_step_kernel<float, NGM, 1, 8, false, 2, 256> "
                                  "at steps 5 and 6, caches flushed, on the build before the search's top "
                                  "levels moved to shuffles (DRAM traffic then 95200768 B a launch)"},
    "sv_fused_step": {"dram_bytes_per_launch": 1156352, "issue_active": 0.397,
                      "source": "ncu dram__bytes_read.sum + dram__bytes_write.sum (caches flushed) and "
                                "smsp__issue_active (warm caches, as in a pass), "
                                "airpf_step_kernel<float, SV, 1, 4, false, 3, 256>"},
    "fp64_ngm_island_step": {"fp64_pipe": 0.858, "issue_active": 0.122,
                             "source": "ncu sm__inst_executed_pipe_fp64 (pct of peak, active cycles), "
                                       "airpf_step_kernel<double, NGM, 1, 4, false, 2, 256>"},
    "fp64_sv_fused_step": {"fp64_pipe": 0.736, "issue_active": 0.110,
                           "source": "ncu sm__inst_executed_pipe_fp64 (pct of peak, active cycles), "
                                     "airpf_step_kernel<double, SV, 1, 4, false, 3, 256>"},
}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def oracle_sample(T_s: int, iter_: int):
    """The CPU oracle on the first T_s observations of the headline workload; returns seconds."""
    import oracle
    y = synth.ngm_observations(T_OBS, seed=5)[:T_s]
    t0 = time.perf_counter()
    oracle.airpf(synth.MODEL_NGM, synth.NGM_THETA, y, m=M_ISL, M=M_PART, mode=oracle.MODE_ADAPTIVE,
                 tau=TAU, seed=1, chain=0, iter=iter_, record=False)
    return time.perf_counter() - t0


def cpu_cores():
    n = os.environ.get("OMP_NUM_THREADS")
    return int(n) if n else (os.cpu_count() or 1)


def calibrate_oracle(target_s: float) -> int:
    t = oracle_sample(2, 0xFFFF0000)
    per_step = max(t / 2, 1e-4)
    return int(max(1, min(T_OBS, target_s / per_step)))


def cpu_baseline_leg(target_s: float = 12.0) -> dict:
    """The oracle on a bounded sample of the headline workload: its first T_s steps, repeated
    over fresh random streams until about target_s seconds of CPU work."""
    T_s = calibrate_oracle(target_s)
    secs, runs = 0.0, 0
    while secs < 0.8 * target_s and runs < 64:
        secs += oracle_sample(T_s, 0xFFFF0001 + runs)
        runs += 1
    return {"value": M_ISL * M_PART * T_s * runs / secs, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
            "sample": f"FP64 oracle (Algorithm 1, stage by stage, OpenMP over islands) on the first {T_s} of "
                      f"{T_OBS} steps of the NGM workload, m={M_ISL} x M={M_PART}, {runs} run(s), {secs:.1f} s"}


def run_reference(args) -> None:
    ws, rank, _ = _dist()
    if rank != 0:
        return
    budget = 150.0
    per_step_target = max(0.5, budget / max(1, args.steps + args.warmup))
    T_s = calibrate_oracle(per_step_target)
    for w in range(args.warmup):
        oracle_sample(T_s, 0xFFFE0000 + w)
    times = [oracle_sample(T_s, j) for j in range(args.steps)]
    tot = sum(times)
    value = M_ISL * M_PART * T_s * args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (NGM observations simulated from seed 5)",
            "config": {"workload": WORKLOAD, "sample_steps": T_s, "note": "each step: the oracle on the "
                       f"first {T_s} observations"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                             "sample": f"first {T_s} of {T_OBS} steps per bench step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def batched_leg(gp, torch, ws: int, n_chains: int = 256, T: int = 500, passes: int = 2) -> dict:
    """Batched serving of proposals: 256 SV chains with their own theta and uneven sizes
    (m in {64, 256, 1024, 4096} x M in {32, 128, 512, 1024}, uniform per chain), T = 500,
    FP32; one context per size class with an autotuned tiling, the classes run side by
    side as a group.  A group pass is one PMMH likelihood evaluation for every chain."""
    ms_, Ms_ = synth.batched_sizes(n_chains, seed=8)
    thetas, redraws = synth.batched_sv_thetas(n_chains, seed=7)
    y = torch.tensor(synth.sv_observations(T, seed=2), device="cuda")
    keys = sorted(set(zip(ms_.tolist(), Ms_.tolist())))
    members, th, c0, base = [], [], [], 0
    t0 = time.perf_counter()
    for (m, M) in keys:
        idx = [i for i in range(n_chains) if (ms_[i], Ms_[i]) == (m, M)]
        tht = torch.tensor(thetas[idx], device="cuda")
        best, _ = gp.autotune(synth.MODEL_SV, tht, y[:16], m=m, M=M, B=len(idx), precision="fp32", seed=1, passes=2)
        members.append(gp.AIRPF(synth.MODEL_SV, m=m, M=M, T=T, B=len(idx), mode="adaptive", tau=TAU,
                                precision="fp32", seed=1, stream=torch.cuda.Stream(), **best))
        th.append(tht)
        c0.append(base)
        base += len(idx)
    tune_s = time.perf_counter() - t0
    grp = gp.Group(members)
    grp.run(th, y, c0, iter=0xFFFF0000)
    grp.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for j in range(passes):
        grp.run(th, y, c0, iter=j)
    e1.record()
    grp.sync()
    torch.cuda.synchronize()
    ms_pass = e0.elapsed_time(e1) / passes
    ps = float((ms_ * Ms_).sum()) * T
    # each class alone on its own stream: the overlap inside a group pass (sum of the classes'
    # times against the group's) and its critical path (the slowest class)
    classes = []
    for (m, M), mb, tht, cb in zip(keys, members, th, c0):
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        mb.run(tht, y, chain0=cb, iter=0xFFFF0001)
        a0.record(mb.stream)
        mb.run(tht, y, chain0=cb, iter=0)
        a1.record(mb.stream)
        mb.sync()
        classes.append({"m": m, "M": M, "chains": mb.B, "ms_alone": a0.elapsed_time(a1), "launch_mode": mb.launch_mode})
    classes.sort(key=lambda r: -r["ms_alone"])
    # the group's roofline: the FP32 path's lane operations per particle-step, with the
    # binary search over each chain's own M (7 per level)
    ops = sum((ops_per_particle_step("SV") - OPS_COMMON["binary_search_M256"] + 7 * np.ceil(np.log2(M))) * m * M * T
              for m, M in zip(ms_.tolist(), Ms_.tolist()))
    peaks, peak_src = _peaks()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    peak = sms * LANES_PER_SM * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    achieved = ops / (ms_pass / 1e3) / 1e12
    out = {"workload": f"batched_sv_{n_chains}chains_T{T}", "particles": int((ms_ * Ms_).sum()),
           "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
                        "note": "all classes' island-step kernels of one group pass"},
           "classes_alone": classes, "sum_of_classes_ms": sum(r["ms_alone"] for r in classes),
           "slowest_class_ms": classes[0]["ms_alone"],
           "classes": len(keys), "ms_per_pass": ms_pass,
           "particle_steps_per_s": ps * ws / (ms_pass / 1e3),
           "chain_iters_per_s": n_chains * ws / (ms_pass / 1e3), "passes": passes,
           "autotune_s": tune_s, "theta_redraws": int(redraws), "precision": "fp32"}
    grp.close()
    for mb in members:
        mb.close()
    return out


def grad_leg(gp, torch, ws: int, passes: int = 2) -> dict:
    """Differentiation workload: LGSSM d_x = 8, d_y = 4 (A = 0.8 I + 0.05 G scaled to spectral
    radius 0.95, C ~ N(0, 1/d_x), Q = 0.1 I, R = 0.5 I), T = 200, m = 2048 x M = 128, FP32;
    one evaluation = the forward pass plus the backward pass (adjoint gradient and Fisher
    score over the 10 parameters), states kept every 10 steps."""
    dx, dy, T = 8, 4, 200
    A, C, md = synth.lg_model(dx, dy, seed=4)
    th = torch.tensor(synth.lg_theta(A, q=0.1, r=0.5)[None, :], device="cuda")
    y = torch.tensor(synth.lg_observations(A, C, 0.1, 0.5, T, seed=4), device="cuda")
    f = gp.AIRPF(synth.MODEL_LGSSM, m=2048, M=128, T=T, B=1, dx=dx, dy=dy, mode="adaptive", tau=TAU,
                 precision="fp32", seed=1, record=gp.RECORD_GRAD, model_data=md, ckpt=10)
    f.grad(th, y, iter=0xFFFF0000)
    f.sync()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record(f.stream)
    for j in range(passes):
        out = f.grad(th, y, iter=j)
    e1.record(f.stream)
    for j in range(passes):
        f.run(th, y, iter=j)
    e2.record(f.stream)
    f.sync()
    ms = e0.elapsed_time(e1) / passes
    ms_fwd = e1.elapsed_time(e2) / passes
    # Langevin-proposal PMMH on the 10 parameters (one gradient pass per iteration)
    n_pm = 4
    st_th, st_lz = th.clone(), torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    st_g = torch.zeros_like(th)
    hstep = [0.002] * dx + [0.01, 0.01]
    lo = list(synth.lg_theta(A, q=0.1, r=0.5) - 1.0)
    hi = list(synth.lg_theta(A, q=0.1, r=0.5) + 1.0)
    f.pmmh_langevin(y, st_th, st_lz, st_g, step=hstep, lo=lo, hi=hi, iters=1, iter0=0)
    f.sync()
    e3, e4 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e3.record(f.stream)
    pm = f.pmmh_langevin(y, st_th, st_lz, st_g, step=hstep, lo=lo, hi=hi, iters=n_pm, iter0=1)
    e4.record(f.stream)
    f.sync()
    ms_pm = e3.elapsed_time(e4) / n_pm
    res = {"workload": "lgssm_dx8_dy4_m2048_M128_T200", "ms_per_eval": ms, "grad_evals_per_s": ws / (ms / 1e3),
           "langevin_pmmh_iters_per_s": ws / (ms_pm / 1e3), "langevin_accepted": int(pm["n_accept"].item()),
           "langevin_iters": n_pm,
           "forward_ms": ms_fwd, "backward_over_forward": (ms - ms_fwd) / ms_fwd, "ckpt": 10,
           "roofline": {"bound": "latency", "kernel": "grad_island_kernel<float, LGSSM, 8>",
                        "backward_ms_per_step": (ms - ms_fwd) / T, "frac": None,
                        "note": "latency: issue active 59-60%, long_scoreboard the top stall (gathers by parent, "
                                "vector atomics to the parents), ncu metrics of grad_island_kernel<float, LGSSM, 8>"},
           "precision": "fp32", "score_norm": float(out["score"].norm()), "grad_norm": float(out["grad"].norm())}
    f.close()
    return res


def ngm_sweep_leg(gp, torch, ws: int, T: int = 1000) -> dict:
    """The large nonlinear-growth workload at the other particle counts of its sweep: m = 65536
    islands, M in {64, 128, 512}, FP32, adaptive tau = 0.3, T = 1000 (one timed pass each,
    after one untimed pass; M = 256 is the headline)."""
    y = torch.tensor(synth.ngm_observations(T, seed=5), device="cuda")
    th = torch.tensor(synth.NGM_THETA[None, :], device="cuda")
    out = {"workload": f"ngm_m65536_T{T}", "points": []}
    for M in (64, 128, 512):
        f = gp.AIRPF(synth.MODEL_NGM, m=65536, M=M, T=T, B=1, mode="adaptive", tau=TAU, precision="fp32", seed=1)
        f.run(th, y, iter=0xFFFF0000)
        f.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(f.stream)
        lz = f.run(th, y, iter=1)["log_z"]
        e1.record(f.stream)
        f.sync()
        ms = e0.elapsed_time(e1)
        out["points"].append({"M": M, "precision": "fp32", "ms_per_pass": ms,
                              "particle_steps_per_s": 65536 * M * T * ws / (ms / 1e3), "log_z": float(lz.item())})
        f.close()
    return out


def kernel_times(gp, torch, model, theta, y, *, m, M, T, prec, passes, flush, chain=0, **tiling):
    """Per-kernel durations of one pass, live: the same workload through a graph with CUDA
    event-record nodes around each kernel of every step (island-step kernel; cascade kernel
    where there is one).  Returns (island us per step, cascade us per step, ms per pass)."""
    ft = gp.AIRPF(model, m=m, M=M, T=T, B=1, mode="adaptive", tau=TAU, precision=prec, seed=1,
                  record=gp.RECORD_TIMING, **tiling)
    ft.run(theta, y, chain0=chain, iter=0xFFFE0000)
    ft.sync()
    isl_ms = cas_ms = pass_ms = 0.0
    for j in range(passes):
        flush.fill_(j & 0xFF)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ft.stream)
        ft.run(theta, y, chain0=chain, iter=j)
        e1.record(ft.stream)
        a, b = ft.kernel_times()
        isl_ms += a
        cas_ms += b
        pass_ms += e0.elapsed_time(e1)
    mode = ft.launch_mode
    ft.close()
    return 1e3 * isl_ms / (passes * T), 1e3 * cas_ms / (passes * T), pass_ms / passes, mode


def alu_roofline(model: str, N: int, step_us: float, sms: int, peaks: dict, peak_src: str) -> dict:
    ops = ops_per_particle_step(model)
    achieved = ops * N / (step_us / 1e6) / 1e12
    peak = sms * LANES_PER_SM * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
            "ops_per_particle_step": ops, "units_per_launch": N, "launch_avg_us": step_us,
            "peak_source": f"{sms} SMs (device property) x {LANES_PER_SM} lanes x sm_max_mhz ({peak_src})"}


def sv_leg(gp, torch, ws, chain, flush, peaks, peak_src, sms, n_fp32=20, n_fp64=10) -> dict:
    """The stochastic-volatility workload (m = 1024 x M = 256, T = 1000, (mu, phi, sigma) =
    (-1, 0.95, 0.3), adaptive tau = 0.3): FP32-mixed and all-FP64 passes on the same random
    streams (the stated log Z error), the fused step kernel's roofline, and PMMH on (mu, phi,
    sigma) with a box prior mu ~ U(-5, 5), phi ~ U(-1, 1), sigma ~ U(0, 2)."""
    y = torch.tensor(synth.sv_observations(T_OBS, seed=2), device="cuda")
    th = torch.tensor(synth.SV_THETA[None, :], device="cuda")
    N = SV_M_ISL * SV_M_PART
    res = {"workload": SV_WORKLOAD}
    lz = {}
    for prec, n in (("fp32", n_fp32), ("fp64", n_fp64)):
        f = gp.AIRPF(synth.MODEL_SV, m=SV_M_ISL, M=SV_M_PART, T=T_OBS, B=1, mode="adaptive", tau=TAU, precision=prec,
                     seed=1)
        for w in range(3):
            f.run(th, y, chain0=chain, iter=0xFFFF0000 + w)
        f.sync()
        tot, out = 0.0, []
        for j in range(n):
            flush.fill_(j & 0xFF)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(f.stream)
            out.append(f.run(th, y, chain0=chain, iter=j)["log_z"])
            e1.record(f.stream)
            f.sync()
            tot += e0.elapsed_time(e1)
        lz[prec] = torch.cat(out).cpu().numpy()
        res[prec] = {"ms_per_pass": tot / n, "particle_steps_per_s": N * T_OBS * ws * n / (tot / 1e3), "passes": n,
                     "launch_mode": f.launch_mode}
        if prec == "fp32":
            # PMMH on (mu, phi, sigma)
            n_pm = 20
            st_th = th.clone()
            st_lz = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            pm_kw = dict(step=[0.05, 0.01, 0.02], lo=[-5.0, -1.0, 0.0], hi=[5.0, 1.0, 2.0], chain0=chain)
            f.pmmh(y, st_th, st_lz, iters=1, iter0=0, **pm_kw)
            f.sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(f.stream)
            pm = f.pmmh(y, st_th, st_lz, iters=n_pm, iter0=1, **pm_kw)
            e1.record(f.stream)
            f.sync()
            res["pmmh"] = {"iters_per_s": n_pm * ws / (e0.elapsed_time(e1) / 1e3), "iters": n_pm,
                           "accepted": int(pm["n_accept"].item()),
                           "proposal": "random walk, steps (0.05, 0.01, 0.02) on (mu, phi, sigma), box prior "
                                       "U(-5,5) x U(-1,1) x U(0,2)"}
        f.close()
    n = min(len(lz["fp32"]), len(lz["fp64"]))
    res["log_z"] = {"fp32_mean": float(lz["fp32"].mean()), "fp32_sd": float(lz["fp32"].std(ddof=1)),
                    "fp64_mean": float(lz["fp64"].mean()), "fp64_sd": float(lz["fp64"].std(ddof=1)),
                    "same_stream_abs_diff_mean": float(np.mean(np.abs(lz["fp32"][:n] - lz["fp64"][:n])))}
    isl, cas, pms, mode = kernel_times(gp, torch, synth.MODEL_SV, th, y, m=SV_M_ISL, M=SV_M_PART, T=T_OBS,
                                       prec="fp32", passes=5, flush=flush, chain=chain, launch="steps")
    step_us = 1e3 * res["fp32"]["ms_per_pass"] / T_OBS
    rf = alu_roofline("SV", N, step_us, sms, peaks, peak_src)
    rf.update({"kernel": "airpf_step_kernel<float, SV, 1, 4, false, 3, 256> (fused step: cascade + island work)",
               "launch_avg_source": "timed passes: pass time / T (one kernel per step and the gaps)",
               "algorithmic_bytes_per_launch": 8 * N,
               "traffic": NCU["sv_fused_step"]["dram_bytes_per_launch"],
               "ncu_issue_active": NCU["sv_fused_step"]["issue_active"], "ncu_source": NCU["sv_fused_step"]["source"],
               "event_nodes": {"step_kernel_us": isl, "ms_per_pass_with_event_nodes": pms}})
    res["roofline"] = rf
    res["fp64"]["roofline"] = {"bound": "fp64", "kernel": "airpf_step_kernel<double, SV, 1, 4, false, 3, 256>",
                               "fp64_pipe_frac_ncu": NCU["fp64_sv_fused_step"]["fp64_pipe"],
                               "ncu_issue_active": NCU["fp64_sv_fused_step"]["issue_active"],
                               "ncu_source": NCU["fp64_sv_fused_step"]["source"],
                               "over_fp32": res["fp64"]["ms_per_pass"] / res["fp32"]["ms_per_pass"]}
    return res


def changepoint_leg(gp, torch, ws: int, T: int = 523) -> dict:
    """Change-point workload of Section 4.2 on synthetic counts: m = 64 islands, M in
    {200, 500}, T = 523, adaptive tau = 0.3; random-walk PMMH on p (step 0.01, U(0, 1)
    prior, alpha and beta fixed), FP32 and FP64, one chain and 256 chains side by side
    (one context, B = 256).  Times PMMH iterations after two untimed ones."""
    y = torch.tensor(synth.cp_observations(T, seed=6), device="cuda")
    a, b = float(synth.CP_THETA[1]), float(synth.CP_THETA[2])
    step, lo, hi = [0.01, 0.0, 0.0], [0.0, a, b], [1.0, a, b]
    out = {"workload": f"changepoint_m64_T{T}", "points": []}
    for M in (200, 500):
        for prec in ("fp32", "fp64"):
            for B in (1, 256):
                f = gp.AIRPF(synth.MODEL_CP, m=64, M=M, T=T, B=B, dy=2, mode="adaptive", tau=TAU, precision=prec,
                             seed=1)
                th = torch.tensor(np.tile(synth.CP_THETA, (B, 1)), device="cuda")
                lz = torch.full((B,), float("nan"), dtype=torch.float64, device="cuda")
                acc = torch.zeros(B, dtype=torch.int32, device="cuda")
                f.pmmh(y, th, lz, step=step, lo=lo, hi=hi, iters=2, chain0=0, iter0=0, n_accept=acc)
                f.sync()
                iters = 40 if B == 1 else 8
                acc.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(f.stream)
                f.pmmh(y, th, lz, step=step, lo=lo, hi=hi, iters=iters, chain0=0, iter0=2, n_accept=acc)
                e1.record(f.stream)
                f.sync()
                ms = e0.elapsed_time(e1)
                out["points"].append({"M": M, "precision": prec, "chains": B, "ms_per_iter": ms / iters,
                                      "pmmh_iters_per_s": B * ws * iters / (ms / 1e3),
                                      "particle_steps_per_s": B * ws * iters * 64 * M * T / (ms / 1e3),
                                      "accept_rate": float(acc.sum().item()) / (B * iters),
                                      "launch_mode": f.launch_mode})
                f.close()
    return out


def run_gpu(args) -> None:
    import torch
    import paper_2312_06484_gb300 as gp
    from paper_2312_06484_gb300 import replicas

    ws, rank, local = replicas.world()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    peaks, peak_src = _peaks()

    prec = args.precision
    y_np = synth.ngm_observations(T_OBS, seed=5)
    theta = torch.tensor(synth.NGM_THETA[None, :], device="cuda")
    y = torch.tensor(y_np, device="cuda")
    tile = dict(ppt=args.ppt, islands_per_cta=args.islands_per_cta)
    f = gp.AIRPF(synth.MODEL_NGM, m=M_ISL, M=M_PART, T=T_OBS, B=1, mode="adaptive", tau=TAU, precision=prec,
                 seed=1, launch=args.launch, **tile)
    launch_name = {1: "fused steps: one kernel per step (CUDA graph, programmatic dependent launch)",
                   2: "persistent, CTA per filter", 3: "persistent cooperative grid",
                   4: "split steps: an island kernel and a group-cascade kernel per step "
                      "(CUDA graph, programmatic dependent launch)"}[f.launch_mode]
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    stream = f.stream
    chain = replicas.chain_base(rank)      # one independent chain per rank

    def one(j):
        return f.run(theta, y, chain0=chain, iter=j)["log_z"]

    for w in range(args.warmup):
        one(0xFFFF0000 + w)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    lzs = []
    clocks = ClockSampler(local)
    clocks.start()
    launches = 0
    for j in range(args.steps):
        flush.fill_(j & 0xFF)                     # L2 flush between timed steps (not timed)
        starts[j].record(stream)
        lzs.append(one(j))
        ends[j].record(stream)
        launches += f.launch_count()
    f.sync()
    clk = clocks.stop()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms = [s_.elapsed_time(e_) for s_, e_ in zip(starts, ends)]
    tot_ms = sum(step_ms)
    tot_ms = replicas.max_over_ranks(tot_ms, device="cuda")   # the slowest rank's time
    N = M_ISL * M_PART
    ps = N * T_OBS
    value = replicas.job_rate(ps * args.steps, tot_ms / 1e3, ws)
    lz32 = torch.cat(lzs).cpu().numpy()

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    th_h = torch.tensor(synth.NGM_THETA[None, :], dtype=torch.float64).pin_memory()
    y_h = torch.tensor(y_np, dtype=torch.float64).pin_memory()
    lz_h = torch.empty(1, dtype=torch.float64).pin_memory()
    n_e2e = max(3, min(args.steps, 10))
    import ctypes
    lib = f.lib
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for j in range(n_e2e):
        st = lib.airpf_run_host(f.ctx, ctypes.c_void_p(th_h.data_ptr()), ctypes.c_void_p(y_h.data_ptr()),
                                chain, 0x10000000 + j, ctypes.c_void_p(lz_h.data_ptr()))
        gp._binding.check(st, f.ctx)
    e2e_s = time.perf_counter() - t0
    e2e = {"value": ps * n_e2e * ws / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 8 * (3 + T_OBS),
           "d2h_bytes_per_step": 8, "steps": n_e2e, "call": "airpf_run_host (host theta, y, log Z)"}

    # the all-FP64 path on the same workload and the same random streams (the stated log Z error)
    fp64 = None
    if not args.no_fp64 and prec != "fp64":
        f64 = gp.AIRPF(synth.MODEL_NGM, m=M_ISL, M=M_PART, T=T_OBS, B=1, mode="adaptive", tau=TAU,
                       precision="fp64", seed=1)
        f64.run(theta, y, chain0=chain, iter=0xFFFF0000)
        f64.sync()
        n64 = 2
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(f64.stream)
        l64 = [f64.run(theta, y, chain0=chain, iter=j)["log_z"] for j in range(n64)]
        e1.record(f64.stream)
        f64.sync()
        ms64 = e0.elapsed_time(e1) / n64
        lz64 = torch.cat(l64).cpu().numpy()
        fp64 = {"workload": WORKLOAD, "value": ps * ws / (ms64 / 1e3), "ms_per_pass": ms64, "passes": n64,
                "over_fp32": ms64 / (tot_ms / args.steps),
                "log_z_fp64": lz64.tolist(), "log_z_fp32_same_streams": lz32[:n64].tolist(),
                "log_z_abs_diff_mean": float(np.mean(np.abs(lz32[:n64] - lz64))),
                "log_z_fp32_sd_over_passes": float(lz32.std(ddof=1)) if lz32.size > 1 else None,
                "roofline": {"bound": "fp64", "kernel": "airpf_step_kernel<double, NGM, 1, 4, false, 2, 256>",
                             "fp64_pipe_frac_ncu": NCU["fp64_ngm_island_step"]["fp64_pipe"],
                             "ncu_issue_active": NCU["fp64_ngm_island_step"]["issue_active"],
                             "ncu_source": NCU["fp64_ngm_island_step"]["source"]}}
        f64.close()

    # per-kernel durations, live (event-record nodes around each kernel)
    isl_us, cas_us, pass_evt_ms, kmode = kernel_times(gp, torch, synth.MODEL_NGM, theta, y, m=M_ISL, M=M_PART,
                                                      T=T_OBS, prec=prec, passes=3, flush=flush, chain=chain,
                                                      launch=args.launch, **tile)

    sv = None if args.no_sv else sv_leg(gp, torch, ws, chain, flush, peaks, peak_src, sms)
    sweep = None if args.no_ngm else ngm_sweep_leg(gp, torch, ws)
    batched = None if args.no_batched else batched_leg(gp, torch, ws)
    gradient = None if args.no_grad else grad_leg(gp, torch, ws)
    changepoint = None if args.no_changepoint else changepoint_leg(gp, torch, ws)

    ms_step = tot_ms / args.steps
    step_us = 1e3 * ms_step / T_OBS           # one time step: the island kernel, the cascade kernel and gaps
    roof = alu_roofline("NGM", N, step_us, sms, peaks, peak_src)
    roof.update({
        "kernel": "airpf_step_kernel<float, NGM, 1, 8, false, 2, 256> (split step: the island launch, then "
                  "airpf_group_cascade_kernel<float, 1>)" if f.launch_mode == 4 else "airpf_step_kernel (one time step)",
        "launch_avg_source": "timed region: pass time / T (a step's island and cascade kernels and the gaps, so "
                             "the island kernel's own fraction is higher by its share of the step)",
        "algorithmic_bytes_per_launch": 8 * N,
        "traffic": NCU["ngm_island_step"]["dram_bytes_per_launch"],
        "ncu_issue_active": NCU["ngm_island_step"]["issue_active"],
        "ncu_source": NCU["ngm_island_step"]["source"],
        "ops_breakdown": {**OPS_COMMON, **OPS_MODEL["NGM"]},
        "event_nodes": {"island_kernel_us": isl_us, "cascade_kernel_us": cas_us,
                        "ms_per_pass_with_event_nodes": pass_evt_ms, "launch_mode": kmode,
                        "note": "events around each kernel in the graph; each interval also holds the "
                                "node-to-node latency, so compare the share with the ncu launch list"}})
    kernels = {"ngm_island_step_fp32": {k: roof[k] for k in ("bound", "frac", "achieved", "peak", "unit")}}
    if fp64:
        kernels["ngm_island_step_fp64"] = fp64["roofline"]
    if sv:
        kernels["sv_fused_step_fp32"] = {k: sv["roofline"][k] for k in ("bound", "frac", "achieved", "peak", "unit")}
        kernels["sv_fused_step_fp64"] = sv["fp64"]["roofline"]
    if batched:
        kernels["batched_group"] = batched.get("roofline")
    if gradient:
        kernels["gradient"] = gradient.get("roofline")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if prec != "fp64" else "f64",
        "data": "synthetic (NGM observations simulated from seed 5)",
        "config": {"workload": WORKLOAD, "model": "NGM", "m": M_ISL, "M": M_PART, "N": N,
                   "T": T_OBS, "interaction": f"adaptive tau={TAU}", "precision": prec,
                   "l2": "flushed between timed steps (256 MiB write, outside the step events); the particle "
                         "stores (2 x 67 MB) exceed L2 as well",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "1 GPU", "launch": launch_name,
                   "sms": sms},
        "pmcmc_iters_per_s": sv["pmmh"]["iters_per_s"] if sv else None,
        "pmcmc_workload": SV_WORKLOAD,
        "filter_passes_per_s": args.steps * ws / (tot_ms / 1e3),
        "log_z": {"mean": float(lz32.mean()), "sd": float(lz32.std(ddof=1)) if lz32.size > 1 else None},
        "clocks": clk,
        "e2e": e2e,
        "gpu_launches": launches,
        "roofline": roof,
        "kernels": kernels,
        "fp64_path": fp64,
        "sv": sv,
        "ngm_sweep": sweep,
        "batched": batched,
        "gradient": gradient,
        "changepoint": changepoint,
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_leg()
    if rank == 0:
        print(json.dumps(line), flush=True)
    f.close()
    if dist:
        dist.destroy_process_group()


def run_stepwise_times() -> None:
    """The m = 65536 x M = 256 NGM pass on a T = 200 series, once from its CUDA graph and once
    step by step through the stepwise ABI with CUDA events around each island and cascade
    launch (plain stream order): how much of the cascade the graph hides."""
    import torch
    import paper_2312_06484_gb300 as gp
    T = 200
    y = torch.tensor(synth.ngm_observations(T, seed=5), device="cuda")
    th = torch.tensor(synth.NGM_THETA[None, :], device="cuda")
    f = gp.AIRPF(synth.MODEL_NGM, m=M_ISL, M=M_PART, T=T, B=1, mode="adaptive", tau=TAU, precision="fp32", seed=1)
    for w in range(2):
        f.run(th, y, iter=w)
    f.sync()
    ev = lambda: torch.cuda.Event(enable_timing=True)
    e0, e1 = ev(), ev()
    e0.record(f.stream)
    f.run(th, y, iter=7)
    e1.record(f.stream)
    f.sync()
    f.step_begin(th, y, iter=7)
    marks = []
    for t in range(1, T + 1):
        a, b, c = ev(), ev(), ev()
        a.record(f.stream)
        f.step_islands(t)
        b.record(f.stream)
        f.step_cascade(t)
        c.record(f.stream)
        marks.append((a, b, c))
    f.step_end()
    f.sync()
    isl = [a.elapsed_time(b) * 1e3 for a, b, _ in marks[1:]]          # steps 2..T
    cas = [b.elapsed_time(c) * 1e3 for _, b, c in marks[1:-1]]
    print(json.dumps({"profile_case": "ngm_stepwise", "T": T, "graph_us_per_step": e0.elapsed_time(e1) * 1e3 / T,
                      "island_us_mean": sum(isl) / len(isl), "island_us_min": min(isl),
                      "cascade_us_mean": sum(cas) / len(cas), "cascade_us_min": min(cas)}), flush=True)
    f.close()


def run_profile_case(args) -> None:
    """One workload for a profiler capture (T = 20): the m = 65536 x M = 256 NGM pass (split
    steps; FP32 or FP64), the m = 1024 x M = 256 SV pass (fused steps; FP32 or FP64), or the
    d_x = 8 gradient evaluation.  Prints the time of the last
    of --steps runs (a capture's timing is not a bench value)."""
    import torch
    import paper_2312_06484_gb300 as gp
    T = 20
    if args.profile_case in ("ngm256", "ngm256_fp64"):
        prec = "fp64" if args.profile_case.endswith("fp64") else "fp32"
        f = gp.AIRPF(synth.MODEL_NGM, m=65536, M=256, T=T, B=1, mode="adaptive", tau=TAU, precision=prec, seed=1)
        y = torch.tensor(synth.ngm_observations(T, seed=5), device="cuda")
        th = torch.tensor(synth.NGM_THETA[None, :], device="cuda")
        run = lambda j: f.run(th, y, iter=j)
    elif args.profile_case in ("sv", "sv_fp64"):
        prec = "fp64" if args.profile_case.endswith("fp64") else "fp32"
        f = gp.AIRPF(synth.MODEL_SV, m=SV_M_ISL, M=SV_M_PART, T=T, B=1, mode="adaptive", tau=TAU, precision=prec,
                     seed=1)
        y = torch.tensor(synth.sv_observations(T, seed=2), device="cuda")
        th = torch.tensor(synth.SV_THETA[None, :], device="cuda")
        run = lambda j: f.run(th, y, iter=j)
    else:
        dx, dy = 8, 4
        A, C, md = synth.lg_model(dx, dy, seed=4)
        th = torch.tensor(synth.lg_theta(A, q=0.1, r=0.5)[None, :], device="cuda")
        y = torch.tensor(synth.lg_observations(A, C, 0.1, 0.5, T, seed=4), device="cuda")
        f = gp.AIRPF(synth.MODEL_LGSSM, m=2048, M=128, T=T, B=1, dx=dx, dy=dy, mode="adaptive", tau=TAU,
                     precision="fp32", seed=1, record=gp.RECORD_GRAD, model_data=md, ckpt=5)
        run = lambda j: f.grad(th, y, iter=j)
    ms = 0.0
    for j in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(f.stream)
        run(j)
        e1.record(f.stream)
        f.sync()
        ms = e0.elapsed_time(e1)
    print(json.dumps({"profile_case": args.profile_case, "T": T, "ms_last_run": ms}), flush=True)
    f.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="airpf", choices=["airpf", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-chains leg")
    ap.add_argument("--no-grad", action="store_true", help="skip the gradient leg")
    ap.add_argument("--no-ngm", action="store_true", help="skip the NGM particle-count sweep")
    ap.add_argument("--no-sv", action="store_true", help="skip the stochastic-volatility leg")
    ap.add_argument("--no-changepoint", action="store_true", help="skip the change-point PMMH leg")
    ap.add_argument("--profile-case", choices=["ngm256", "ngm256_fp64", "sv", "sv_fp64", "grad", "ngm_stepwise"],
                    default=None,
                    help="run one small workload for a profiler capture instead of the bench line")
    ap.add_argument("--launch", default="auto", choices=["auto", "steps", "split", "grid"])
    ap.add_argument("--ppt", type=int, default=0, help="particles per thread (0: automatic)")
    ap.add_argument("--islands-per-cta", type=int, default=0, help="islands per CTA (0: automatic)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("at least 3 warm-up steps")
    if args.impl == "reference":
        run_reference(args)
    elif args.profile_case == "ngm_stepwise":
        run_stepwise_times()
    elif args.profile_case:
        run_profile_case(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
