#!/usr/bin/env python3
"""Benchmark of the BSS-MPPI hot path: particle-steps/s of one controller's solve step.

A step is one pass of the whole path on the racing workload K=4096 control samples, M=64
particles, T=40 steps (6-state dynamic bicycle, 5 Euler substeps): control noise, clamp,
disturbance draws, particle rollout, per-step belief moments, barrier and cost, then weights,
update and the warm-start shift in the same kernel's tail (one launch per step). Inputs are resident on the device;
the L2 cache is flushed (a 256 MiB write) before every timed step, outside the timed events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]
                  [--mode replicas|shard]

Prints one JSON line. With N > 1 (launched under torchrun, or re-launched under it by this script
when started without one) every rank solves its own controller in the default mode (replicas on
independent tracks; no collective on the data path) and rank 0 prints the whole-job throughput
from the slowest rank's time. `--mode shard` instead splits one solve's K samples over the ranks
(one all-gather of the 3 + 2T log-sum-exp partials per solve): strong scaling of one solve.
`--impl reference` times the FP64 oracle on the host cores instead.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workload  # noqa: E402

METRIC = "particle-steps/s (K*M*T per solve)"
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one rollout_kernel launch, from one
# ncu capture of the current kernel on each workload (None where none was taken).
ROLLOUT_DRAM_BYTES = {"racing_K4096_M64_T40": 126976}
# Device facts for the nominal ALU peak (GB300: 152 SMs, 128 FP32 lanes per SM, max SM clock); the
# roofline's denominator is the FP32 peak measured on the device in the same run (bssmppi_fp32_peak).
SMS, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0
# Issue-slot and FMA-pipe activity of the rollout kernel from the committed ncu capture of the
# current kernel (sm__inst_executed.avg.per_cycle_active / 4 and the FMA pipe's share of its peak).
ROLLOUT_NCU = {"racing_K4096_M64_T40": {"issue_slots_busy": 2.85 / 4, "fma_pipe_of_peak": 0.401,
                                        "lane_instructions_per_particle_step": 691,
                                        "source": "profiles/rollout_kernel_racing_K4096_M64_T40.md"}}


def algorithmic_flops_per_particle_step(prob) -> float:
    """FP32-equivalent operations the method needs per particle-step (one particle, one dt).

    Counting convention: add, sub, mul, min, max, compare, floor and each integer Philox operation
    = 1; fma = 2; division, reciprocal, square root = 4; each of exp, log, sin, cos, atan = 8
    (sincos = 16). Counted from the method's formulas (model, noise, moments), not from any kernel.
    """
    if prob.model == workload.MODEL_BICYCLE6:
        # per Euler substep: floor on v_x 1, 1/v_x 4, front/rear slip 2x(2 + 1 + 8 + 1),
        # two tyre forces 2x(1 + 8 + 1 + 8 + 1), curvature lookup 7, sincos(e_psi) 16,
        # s' 9, v_x' 5, v_y' 5, r' 5, e_psi' 2, e_y' 3, six Euler fmas 12
        substep = 1 + 4 + 2 * 12 + 2 * 19 + 7 + 16 + 9 + 5 + 5 + 5 + 2 + 3 + 12
        model = prob.n_sub * substep
        nx = 6
    else:
        model = 4 * 2 + 2 * 2  # exact ZOH step: 4 + 2 fmas
        nx = 4
    pairs = (nx + 1) // 2
    philox_calls = pairs / 2              # nx Gaussians need nx uniform words: a call gives four
    philox = philox_calls * 10 * 10       # 10 rounds x (2 wide multiplies = 4, 2 three-way xors = 4, 2 key adds)
    box_muller = pairs * (2 + 8 + 1 + 4 + 16 + 2)
    disturbance = nx * (nx + 1) // 2 * 2 + nx  # L_w z (fmas) and x += w
    moments = 2 * nx + 3                   # mean sums and the e_y second moment
    return float(model + philox + box_muller + disturbance + moments)


# ------------------------------------------------------------------------------------------------
def _problem(name: str, rank: int = 0):
    if name == "racing_K4096_M64_T40":
        p = workload.config1()
    elif name == "racing_K256_M16_T20":
        p = workload.config0()
    elif name == "racing_K16384_M128_T60":
        p = workload.config3(1.0)
    else:
        raise SystemExit(f"unknown workload {name}")
    p.seed = int(p.seed) + 1000 * rank  # replicas: independent random streams per rank
    return p


def _workload_desc(p, name):
    return {"workload": name, "K": p.K, "M": p.M, "T": p.T, "model": "dynamic bicycle (6 states)",
            "n_sub": p.n_sub, "track": "seeded Fourier-perturbed circle, R=60 m, half-width 3 m",
            "l2": "flushed before every timed step (256 MiB device write, outside the timed events)"}


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 8:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------------------------------------
def cpu_model() -> str:
    """The host CPU's model name (lscpu), or the machine type."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.TimeoutExpired):
        pass
    import platform
    return platform.machine()


def _time_oracle(p, threads, budget_s):
    """Rollout and cost of the first k samples of one solve, k sized to about budget_s seconds."""
    import oracle

    o = oracle.Oracle(p)
    x0 = workload.racing_x0(p)
    v = np.zeros((p.T, 2), np.float32)
    k = min(p.K, 8 * threads)
    t0 = time.perf_counter()
    o.solve(x0, v, 0, k_range=(0, k), threads=threads)
    dt = time.perf_counter() - t0
    k = int(min(p.K, max(k, k * budget_s / max(dt, 1e-6))))
    t0 = time.perf_counter()
    o.solve(x0, v, 0, k_range=(0, k), threads=threads)
    dt = time.perf_counter() - t0
    return k, dt


def run_cpu_baseline(p, budget_s: float = 12.0):
    """The FP64 oracle as it stands on a bounded sample of the same solve: on all host cores (the
    line's value; OpenMP threads over samples) and on one thread."""
    import oracle

    threads = oracle.host_threads()
    k1, dt1 = _time_oracle(p, 1, budget_s / 2)
    kn, dtn = _time_oracle(p, threads, budget_s / 2)
    return {"value": kn * p.M * p.T / dtn, "unit": "particle-steps/s", "cores": threads, "kind": "oracle",
            "cpu": cpu_model(),
            "sample": f"rollout and cost of the first {kn} of the {p.K} control samples of one solve "
                      f"({kn * p.M * p.T} particle-steps, {dtn:.1f} s, FP64, {threads} threads)",
            "one_thread": {"value": k1 * p.M * p.T / dt1, "cores": 1,
                           "sample": f"the first {k1} control samples ({k1 * p.M * p.T} particle-steps, "
                                     f"{dt1:.1f} s, FP64, 1 thread)"}}


def run_reference(args):
    """--impl reference: the FP64 oracle on the host cores, a bounded sample of the workload per step."""
    import oracle

    p = _problem(args.workload)
    o = oracle.Oracle(p)
    x0 = workload.racing_x0(p)
    v = np.zeros((p.T, 2), np.float32)
    k_step = max(1, min(p.K, args.ref_samples))
    threads = oracle.host_threads()
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        r = o.solve(x0, v, i, k_range=(0, k_step), threads=threads)
        oracle.optimal_control(r["S"][:k_step], r["u"][:k_step], float(p.lam))
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    mean_s = statistics.fmean(times)
    value = k_step * p.M * p.T / mean_s
    sample = (f"each step: rollout, cost, weights and update of the first {k_step} of the {p.K} control "
              f"samples of one solve ({k_step * p.M * p.T} particle-steps), FP64, {threads} threads")
    return {"metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": mean_s * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": _workload_desc(p, args.workload),
            "cpu_baseline": {"value": value, "unit": "particle-steps/s", "cores": threads, "kind": "oracle",
                             "cpu": cpu_model(), "sample": sample},
            "e2e": {"value": value, "unit": "particle-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


SERVE_BATCH_WORK = 20_000_000  # particle-steps per batch: under 1 ms of GPU time
SERVE_SLOTS = 8                # batches in flight


def _serve_stream(bssmppi, n_ctrl, rate_hz, duration_s, seed, batched, probs_params, batch_work=SERVE_BATCH_WORK,
                  slots=SERVE_SLOTS):
    """Replay a Poisson arrival stream against a server; returns latency/throughput statistics."""
    reqs = workload.serving_requests(n_ctrl=n_ctrl, rate_hz=rate_hz, duration_s=duration_s, seed=seed)
    if batched:
        s = bssmppi.server_create(n_ctrl, max_batch=512, T_max=60, slots=slots, use_graphs=True,
                                  hbm_budget_bytes=2 << 30, max_batch_work=int(batch_work))
    else:
        s = bssmppi.server_create(n_ctrl, max_batch=1, T_max=60, slots=1, use_graphs=False,
                                  hbm_budget_bytes=2 << 30)
    try:
        for prm in probs_params:
            bssmppi.server_add_controller(s, prm)
        x0 = np.array([10.0, 0.0, 0.0, 0.0, 0.0, 5.0], np.float32)
        t0 = time.perf_counter()
        for j, (ta, c, K, M, T) in enumerate(reqs):
            while time.perf_counter() - t0 < ta:
                pass
            bssmppi.server_submit(s, c, x0, K, M, T, req_id=j)
        t_sub = time.perf_counter() - t0
        bssmppi.server_drain(s, 600000)
        t_all = time.perf_counter() - t0
        res = bssmppi.server_poll(s, max_n=len(reqs) + 16)
        stats = bssmppi.server_get_stats(s)
    finally:
        bssmppi.server_destroy(s)
    ok = [r for r in res if r.status == 0]
    lat = np.array([r.t_done_us - r.t_submit_us for r in ok]) * 1e-3
    cls = np.array([r.t_done_us - r.t_submit_us for r in ok if (r.K, r.M, r.T) == (4096, 64, 40)]) * 1e-3
    work = sum(r.K * r.M * r.T for r in ok)
    span = (max(r.t_done_us for r in ok) - min(r.t_submit_us for r in res)) * 1e-6 if ok else float("nan")
    pct = lambda a, q: float(np.percentile(a, q)) if a.size else None
    return {"offered_req_per_s": len(reqs) / duration_s, "submitted": stats["submitted"],
            "completed": len(ok), "replaced_by_newer": stats["superseded"],
            "shed_fraction": stats["superseded"] / max(1, stats["submitted"]), "batches": stats["batches"],
            "max_batch": stats["max_batch_seen"], "solves_per_s": len(ok) / span,
            "particle_steps_per_s": work / span, "latency_ms_p50": pct(lat, 50), "latency_ms_p99": pct(lat, 99),
            "class_4096_64_40_latency_ms_p50": pct(cls, 50), "class_4096_64_40_latency_ms_p99": pct(cls, 99),
            "class_4096_64_40_completed": int(cls.size), "submit_window_s": t_sub, "wall_s": t_all,
            "_class_latencies_ms": cls}


def _sweep_rate(bssmppi, n_ctrl, rate, seconds, repeats, batched, params, bw, slots=SERVE_SLOTS):
    """One rate of the sweep: `repeats` windows of `seconds` each on independent arrival streams
    (seeds 5, 6, ...). The K=4096, M=64, T=40 class's p99 is taken over the pooled latencies of all
    windows; throughput is reported as the mean and range over the windows."""
    runs = [_serve_stream(bssmppi, n_ctrl, rate, seconds, 5 + r, batched, params, bw, slots) for r in range(repeats)]
    pooled = np.concatenate([r.pop("_class_latencies_ms") for r in runs])
    sps = [r["solves_per_s"] for r in runs]
    p99_each = [r["class_4096_64_40_latency_ms_p99"] for r in runs]
    submitted = sum(r["submitted"] for r in runs)
    shed = sum(r["replaced_by_newer"] for r in runs)
    return {"rate_hz_per_controller": rate, "windows": repeats, "window_s": seconds,
            "offered_req_per_s": statistics.fmean(r["offered_req_per_s"] for r in runs),
            "solves_per_s": statistics.fmean(sps), "solves_per_s_min": min(sps), "solves_per_s_max": max(sps),
            "latency_ms_p99_mean_of_windows": statistics.fmean(r["latency_ms_p99"] for r in runs),
            "class_4096_64_40_latency_ms_p99": float(np.percentile(pooled, 99)) if pooled.size else None,
            "class_4096_64_40_latency_ms_p99_per_window": p99_each,
            "class_4096_64_40_completed": int(pooled.size),
            "replaced_by_newer": shed, "shed_fraction": shed / max(1, submitted)}


def solve_kernel_on_the_mix(bssmppi, prm0, K=8192, reps=20):
    """The single-solve kernel's particle-steps/s on each (M, T) class of the serving mix at K=8192
    (one solve + shift per launch, back to back), and the rate it would sustain on the mix's work:
    the work-weighted harmonic mean over the uniform (K, M, T) classes. The server's saturation
    throughput is compared with it."""
    import ctypes

    import torch

    rates = {}
    for M in workload.SERVE_M:
        for T in workload.SERVE_T:
            prm = bssmppi.Params()
            ctypes.pointer(prm)[0] = prm0
            prm.K, prm.M, prm.T = K, M, T
            h = bssmppi.create(prm)
            try:
                x0 = torch.as_tensor(np.array([10.0, 0.0, 0.0, 0.0, 0.0, 5.0], np.float32), device="cuda")
                for _ in range(3):
                    bssmppi.solve_shift(h, x0, None, None, 1)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                for _ in range(reps):
                    bssmppi.solve_shift(h, x0, None, None, 1)
                b.record()
                torch.cuda.synchronize()
                rates[(M, T)] = K * M * T * reps / (a.elapsed_time(b) * 1e-3)
            finally:
                bssmppi.destroy(h)
    kbar = statistics.fmean(workload.SERVE_K)
    work = {c: kbar * c[0] * c[1] for c in rates}
    mix = sum(work.values()) / sum(work[c] / rates[c] for c in rates)
    return {"K": K, "particle_steps_per_s_by_M_T": {f"M{m}_T{t}": r for (m, t), r in rates.items()},
            "mix_particle_steps_per_s": mix,
            "note": "work-weighted harmonic mean over the uniform (K, M, T) mix: the rate one solve at a time "
                    "would sustain with every launch as full as K=8192 makes it"}


def run_serving(args):
    """Serving: 512 controllers on independent tracks, Poisson arrivals at 20 Hz each, (K, M, T)
    drawn from {512, 2048, 4096, 8192} x {8, 32, 64, 128} x {20, 40, 60}; the batched server against
    the one-solve-at-a-time path on the same arrival stream, and a rate sweep."""
    from paper_2408_00494_gb300 import bssmppi

    n_ctrl = 512
    params = []
    for i in range(n_ctrl):
        kappa, length = workload.make_track(1000 + i, n_theta=1 << 12)
        p = workload.racing_problem(256, 16, 20, track_seed=0, noise_scale=2.0, seed=10_000 + i)
        p.kappa, p.track_len = kappa, length
        params.append(bssmppi.make_params(p))
    out = {"controllers": n_ctrl, "rate_hz_per_controller": 20.0, "duration_s": args.serve_seconds,
           "policy": "latest state wins: a newer request of a controller replaces its pending one"}
    bw = args.serve_batch_work
    out["batch_work_limit_particle_steps"] = bw
    out["slots"] = args.serve_slots
    for name, batched in (("batched", True), ("plain", False)):
        r = _serve_stream(bssmppi, n_ctrl, 20.0, args.serve_seconds, 4, batched, params, bw, args.serve_slots)
        r.pop("_class_latencies_ms")
        out[name] = r
    # rate sweep of both paths on the same arrival streams: the highest sustained solves/s at which
    # the K=4096, M=64, T=40 class keeps its p99 latency under 10 ms with at most 1 % of requests shed
    for name, batched in (("batched", True), ("plain", False)):
        sweep, best = [], None
        for rate in args.serve_rates:
            r = _sweep_rate(bssmppi, n_ctrl, rate, args.serve_sweep_seconds, args.serve_repeats, batched, params, bw,
                            args.serve_slots)
            sweep.append(r)
            p99 = r["class_4096_64_40_latency_ms_p99"]
            if p99 is not None and p99 < 10.0 and r["shed_fraction"] <= 0.01:
                best = {k: r[k] for k in ("rate_hz_per_controller", "solves_per_s", "solves_per_s_min",
                                          "solves_per_s_max", "class_4096_64_40_latency_ms_p99",
                                          "class_4096_64_40_completed", "shed_fraction")}
            elif p99 is not None and p99 > 50.0:
                break
        out[f"rate_sweep_{name}"] = sweep
        out[f"{name}_max_solves_per_s_with_p99_under_10ms"] = best
    out["solve_kernel_on_the_mix"] = solve_kernel_on_the_mix(bssmppi, params[0])
    b, q = out["batched_max_solves_per_s_with_p99_under_10ms"], out["plain_max_solves_per_s_with_p99_under_10ms"]
    if b and q:
        out["batched_over_plain_at_p99_under_10ms"] = {
            "ratio": b["solves_per_s"] / q["solves_per_s"],
            "ratio_range": [b["solves_per_s_min"] / q["solves_per_s_max"], b["solves_per_s_max"] / q["solves_per_s_min"]]}
    return out


def run_closed_loop(bssmppi, p, dev, stream, steps: int, seed: int = 1):
    """Closed loop: every step solves from the plant state, applies u0 to the plant (the same model,
    stepped on the device, plus a seeded disturbance drawn with Sigma_w) and shifts the nominal.
    Reports the constraint-violation rate (|e_y| > w_T), the near-violation rate (|e_y| > 0.9 w_T),
    the fraction of steps satisfying the DCBF condition h_{k+1} >= (1 - gamma) h_k with
    h = w_T^2 - e_y^2 on the executed states, and the time per closed-loop step."""
    import torch

    ctl = bssmppi.Controller(p, stream=stream)
    try:
        u0 = torch.zeros(1, 2, device=dev)
        rng = np.random.default_rng(seed)
        std = np.sqrt(np.diag(np.asarray(p.Sigma_w)))
        W = torch.as_tensor((rng.standard_normal((steps, 6)) * std).astype(np.float32), device=dev)
        traj = torch.empty(steps + 1, 6, device=dev)
        traj[0] = torch.as_tensor(workload.racing_x0(p), device=dev)
        bssmppi.timing(ctl.h, min(steps, 4096))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(steps):  # only library calls inside the loop
            bssmppi.solve_shift(ctl.h, traj[k], None, u0[0], 1)
            bssmppi.model_step(ctl.h, traj[k:k + 1], u0, traj[k + 1:k + 2], W[k:k + 1])
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        roll_ms, _ = bssmppi.timing_read(ctl.h, min(steps, 4096))
        bssmppi.timing(ctl.h, 0)
        ey = traj[:, 4].double().cpu().numpy()
        s = traj[:, 5].double().cpu().numpy()
        vx = traj[:, 0].double().cpu().numpy()
    finally:
        ctl.close()
    wT, g = float(p.w_T), float(p.gamma)
    h = wT * wT - ey * ey
    return {"steps": steps, "ms_per_step": dt * 1e3 / steps,
            "solve_kernel_ms_mean": float(np.mean(roll_ms)), "solve_kernel_ms_max": float(np.max(roll_ms)),
            "violation_rate": float(np.mean(np.abs(ey[1:]) > wT)),
            "near_violation_rate": float(np.mean(np.abs(ey[1:]) > 0.9 * wT)),
            "dcbf_condition_satisfied": float(np.mean(h[1:] >= (1.0 - g) * h[:-1])),
            "max_abs_e_y_m": float(np.abs(ey).max()), "distance_m": float(s[-1] - s[0]),
            "mean_speed_mps": float(vx.mean()),
            "plant": "same bicycle model stepped on the device (bssmppi_model_step) + N(0, Sigma_w) per step "
                     "(numpy generator, seed 1, drawn before the loop)"}


def run_km_sweep(bssmppi, dev, stream, Ks, Ms, runs, T=20, noise_scale=4.0, v_goal=10.0, w_T=2.0,
                 collide_at=1.8, seed0=100, q_ey=(0.1,)):
    """Monte-Carlo laps over a grid of sample counts K and particle counts M (Sec. "Simulation
    Results": crash and collision rates versus the number of control sequences and of uncertainty
    trajectories). Each run starts from a seeded state near the centre line at a random lap position,
    drives one lap in closed loop (solve, apply u0 to the plant stepped on the device with a seeded
    N(0, Sigma_w) disturbance, shift) and is scored on the executed states: a crash is |e_y| > w_T
    (the run ends there), a collision is an entry into |e_y| > collide_at. Rates are per run; the
    collision rate can exceed 1."""
    import torch

    out = []
    cells = [(q, K, M) for q in q_ey for K in Ks for M in Ms]
    for qe, K, M in cells:
        crashes = collisions = 0
        dcbf_ok = dcbf_n = 0
        step_s, laps_s = [], []
        for r in range(runs):
            p = workload.racing_problem(K, M, T, track_seed=1, noise_scale=noise_scale, lam=1.0,
                                        seed=seed0 + r, w_T=w_T,
                                        x_goal=(v_goal, 0.0, 0.0, 0.0, 0.0, 0.0),
                                        Q=(1.0, 0.0, 0.0, 1.0, qe, 0.0), Qf=(1.0, 0.0, 0.0, 1.0, qe, 0.0))
            rng = np.random.default_rng(seed0 + r)
            x0 = np.array([v_goal * rng.uniform(0.9, 1.0), 0.0, 0.0, rng.normal(0.0, 0.02),
                           rng.uniform(-0.5, 0.5), rng.uniform(0.0, p.track_len)], np.float32)
            steps = int(1.25 * p.track_len / (v_goal * p.dt)) + 1
            std = np.sqrt(np.diag(np.asarray(p.Sigma_w)))
            W = torch.as_tensor((rng.standard_normal((steps, 6)) * std).astype(np.float32), device=dev)
            traj = torch.empty(steps + 1, 6, device=dev)
            traj[0] = torch.as_tensor(x0, device=dev)
            u0 = torch.zeros(1, 2, device=dev)
            ctl = bssmppi.Controller(p, stream=stream)
            try:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for k in range(steps):
                    bssmppi.solve_shift(ctl.h, traj[k], None, u0[0], 1)
                    bssmppi.model_step(ctl.h, traj[k:k + 1], u0, traj[k + 1:k + 2], W[k:k + 1])
                torch.cuda.synchronize()
                step_s.append((time.perf_counter() - t0) / steps)
            finally:
                ctl.close()
            x = traj.double().cpu().numpy()
            ey, ds = x[:, 4], x[:, 5] - x[0, 5]
            lap = np.nonzero(ds >= p.track_len)[0]
            end = int(lap[0]) if lap.size else steps
            out_of = np.nonzero(~(np.abs(ey[: end + 1]) <= w_T))[0]  # NaN counts as a crash
            if out_of.size:
                crashes += 1
                end = int(out_of[0])
            else:
                laps_s.append(end * p.dt)
            near = np.abs(ey[: end + 1]) > collide_at
            collisions += int(near[0]) + int(np.count_nonzero(near[1:] & ~near[:-1]))
            h = w_T * w_T - ey[: end + 1] ** 2
            dcbf_ok += int(np.count_nonzero(h[1:] >= (1.0 - p.gamma) * h[:-1]))
            dcbf_n += max(end, 0)
        out.append({"q_ey": qe, "K": K, "M": M, "runs": runs, "crash_rate": crashes / runs,
                    "collision_rate": collisions / runs,
                    "dcbf_condition_satisfied": dcbf_ok / max(dcbf_n, 1),
                    "mean_lap_time_s": float(np.mean(laps_s)) if laps_s else None,
                    "ms_per_closed_loop_step": 1e3 * float(np.mean(step_s))})
    return {"T": T, "noise_scale": noise_scale, "v_goal": v_goal, "w_T": w_T, "collide_at": collide_at,
            "track": "seeded Fourier-perturbed circle (track seed 1), one lap per run", "grid": out}


def reduce_over_ranks(values, device, world):
    """Element-wise MAX of per-rank values across the job (identity on one rank)."""
    import torch

    t = torch.tensor(values, dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return t.tolist()


def whole_job_throughput(units_per_rank, slowest_ms, world):
    """Units processed by all ranks per second of the slowest rank."""
    return world * units_per_rank / (slowest_ms * 1e-3)


def run_ours(args, rank, world, local_rank):
    import torch

    from paper_2408_00494_gb300 import bssmppi

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    p = _problem(args.workload, rank)
    ctl = bssmppi.Controller(p, stream=stream)
    h = ctl.h
    x0 = torch.as_tensor(workload.racing_x0(p), device=dev)
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)  # 256 MiB > 129 MB L2

    def step():
        bssmppi.solve_shift(h, x0, None, None, 1)  # solve + warm-start shift of the resident nominal, one launch

    # the roofline's denominator: this device's FP32 multiply-add rate, measured before the timed
    # region (scalar and packed .f32x2 forms; the larger counts)
    peaks = [bssmppi.fp32_peak(packed, 1 << 16, stream) for packed in (False, True)]
    peak_meas = max(peaks, key=lambda r: r["tflops"])
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local_rank)
    clocks.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    bssmppi.timing(h, args.steps)
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    roll_ms, _ = bssmppi.timing_read(h, args.steps)
    bssmppi.timing(h, 0)

    # Shield repair on top: solve + 5 projected-gradient steps of the adjoint kernel + shift
    rep_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for i in range(args.warmup + args.steps):
        flush.fill_(float(i))
        if i >= args.warmup:
            rep_ev[i - args.warmup][0].record(stream)
        bssmppi.solve(h, x0)
        bssmppi.repair(h, x0, None, args.repair_iters, args.repair_step)
        bssmppi.shift(h, None, 1)
        if i >= args.warmup:
            rep_ev[i - args.warmup][1].record(stream)
    torch.cuda.synchronize()
    rep_ms = statistics.fmean(a.elapsed_time(b) for a, b in rep_ev)

    def time_variant(pv, xv=None):
        """Solve + shift of a problem variant from state xv (default: the benchmark's), same L2 flush."""
        xv = x0 if xv is None else xv
        cv = bssmppi.Controller(pv, stream=stream)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for i in range(args.warmup + args.steps):
            flush.fill_(float(i))
            if i >= args.warmup:
                ev[i - args.warmup][0].record(stream)
            bssmppi.solve_shift(cv.h, xv, None, None, 1)
            if i >= args.warmup:
                ev[i - args.warmup][1].record(stream)
        torch.cuda.synchronize()
        cv.close()
        return statistics.fmean(a.elapsed_time(b) for a, b in ev)

    # the literal reading of Algorithm 2 (particles re-drawn from N(mean, cov) before every step)
    p_rs = _problem(args.workload, rank)
    p_rs.resample = 1
    rs_ms = time_variant(p_rs)
    # the general constraint set: track edges as two half-spaces and a disk obstacle 6 m ahead
    p_con = _problem(args.workload, rank)
    x0_np = workload.racing_x0(p_con)
    p_con.constraints = (workload.halfspace((0, 0, 0, 0, 1, 0), p_con.w_T, p_con.delta),
                         workload.halfspace((0, 0, 0, 0, -1, 0), p_con.w_T, p_con.delta),
                         workload.disk(5, 4, (float(x0_np[5]) + 6.0, 0.3), 1.0, 0.05, backoff="cantelli"))
    con_ms = time_variant(p_con)
    # the 8-state single-track model with wheel speeds and combined slip (n_sub = 10), same sizes
    p_w8 = workload.wheels_problem(p.K, p.M, p.T, seed=int(p.seed))
    w8_ms = time_variant(p_w8, torch.as_tensor(workload.racing_x0(p_w8), device=dev))

    # end to end through the C ABI with host buffers (H2D of the state and nominal, D2H of v+ and u0)
    x0_h = workload.racing_x0(p)
    v_h = np.zeros((p.T, 2), np.float32)
    u0_h = np.zeros(2, np.float32)
    e2e_s = []
    for i in range(args.warmup + args.steps):
        flush.fill_(float(i))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bssmppi.solve_host(h, x0_h, None, v_h, u0_h)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            e2e_s.append(dt)
    ctl.close()

    mean_ms = statistics.fmean(step_ms)
    mean_roll = statistics.fmean(roll_ms)
    mean_e2e = statistics.fmean(e2e_s)
    mean_ms, mean_roll, mean_e2e_ms, t_wall = reduce_over_ranks([mean_ms, mean_roll, mean_e2e * 1e3, t_wall], dev, world)
    units = p.K * p.M * p.T
    value = whole_job_throughput(units, mean_ms, world)
    flops = algorithmic_flops_per_particle_step(p) * units
    peak_nominal = SMS * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12
    peak = peak_meas["tflops"]
    achieved = flops / (mean_roll * 1e-3) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": mean_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": _workload_desc(p, args.workload),
        "solves_per_s": world * 1e3 / mean_ms,
        "phases_ms": {"rollout_and_update_kernel": mean_roll},
        "roofline": {"bound": "alu", "kernel": "rollout_kernel", "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": ROLLOUT_DRAM_BYTES.get(args.workload),
                     "peak_basis": (f"measured in this run: FP32 multiply-add microbenchmark (bssmppi_fp32_peak, "
                                    f"{'packed .f32x2' if peak_meas['packed'] else 'scalar'} form, "
                                    f"{peak_meas['sms']} SMs); scalar {peaks[0]['tflops']:.2f}, packed "
                                    f"{peaks[1]['tflops']:.2f} TFLOP/s"),
                     "peak_nominal": peak_nominal, "frac_of_nominal": achieved / peak_nominal,
                     "peak_nominal_basis": "152 SMs x 128 FP32 lanes x 2 (fma) x 2070 MHz max SM clock",
                     "flops_per_particle_step": algorithmic_flops_per_particle_step(p),
                     "ncu": ROLLOUT_NCU.get(args.workload)},
        "e2e": {"value": whole_job_throughput(units, mean_e2e_ms, world), "unit": "particle-steps/s",
                "h2d_bytes_per_step": 4 * (8 + 2 * p.T), "d2h_bytes_per_step": 4 * (2 * p.T + 2),
                "copies_per_step": "one H2D (x0 padded to 8 floats | v) and one D2H (v+ | u0)"},
        "gpu_launches": args.steps,  # per step: one kernel (solve, update and shift fused)
        "resample_variant": {"ms_per_step": rs_ms, "particle_steps_per_s": units / (rs_ms * 1e-3),
                             "note": "Algorithm 2 read literally: full moments, Cholesky and re-draw of "
                                     "every particle before each step; solve + shift in one launch, same L2 flush"},
        "wheels8_variant": {"ms_per_step": w8_ms, "particle_steps_per_s": units / (w8_ms * 1e-3),
                            "note": "8-state single-track model with wheel speeds and friction-ellipse "
                                    "combined slip, n_sub = 10, AutoRally scale; solve + shift in one launch"},
        "constraint_set_variant": {"ms_per_step": con_ms, "particle_steps_per_s": units / (con_ms * 1e-3),
                                   "note": "general set h = min_q h_q: two track-edge half-spaces and a disk "
                                           "obstacle on (s, e_y), full covariance every step; solve + shift in one launch"},
        "shield_repair": {"iters": args.repair_iters, "step": args.repair_step, "ms_per_step": rep_ms,
                          "repair_ms": rep_ms - mean_ms, "solves_per_s": 1e3 / rep_ms,
                          "particle_steps_per_s": units / (rep_ms * 1e-3),
                          "note": "solve + adjoint repair (one launch) + shift per step, same L2 flush"},
        "clocks": clk,
        "wall_s_timed_region": t_wall,
    }
    if rank == 0 and args.closed_loop_steps > 0:
        line["closed_loop"] = run_closed_loop(bssmppi, _problem(args.workload), dev, stream, args.closed_loop_steps)
        # the same loop where the workload's own disturbance never brings the car near the wall:
        # disturbance x6, half-width 2 m, goal 12 m/s (the lap study's track and costs), with the
        # benchmark's 64 particles per sample and with 4
        stress = {}
        for M in (64, 4):
            ps = workload.racing_problem(4096, M, 40, track_seed=1, noise_scale=6.0, lam=1.0, seed=1, w_T=2.0,
                                         x_goal=(12.0, 0.0, 0.0, 0.0, 0.0, 0.0))
            stress[f"M{M}"] = run_closed_loop(bssmppi, ps, dev, stream, args.closed_loop_steps)
            stress[f"M{M}"].pop("plant", None)
        stress["setting"] = ("K=4096, T=40, disturbance std x6 of the small workload's, w_T = 2 m, goal 12 m/s, "
                             "track seed 1; plant as in closed_loop")
        line["closed_loop_stress"] = stress
    if rank == 0 and world == 1 and not args.no_serving:
        line["serving"] = run_serving(args)
    if rank == 0 and args.km_sweep:
        ks, ms = (tuple(int(v) for v in part.split(",")) for part in args.km_sweep.split(";"))
        line["km_sweep"] = run_km_sweep(bssmppi, dev, stream, ks, ms, args.km_runs, T=args.km_T,
                                        noise_scale=args.km_noise, v_goal=args.km_speed, w_T=args.km_wT,
                                        q_ey=tuple(float(q) for q in args.km_qey.split(",")))
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = run_cpu_baseline(p, args.cpu_budget)
    return line


def run_shard(args, rank, world, local_rank):
    """One solve split over the ranks by its K samples (strong scaling): each rank's handle covers
    K/N samples (bssmppi_set_sample_range; the random streams are keyed by the global sample index,
    so the split does not change any sample), rolls them out and reduces them to a log-sum-exp partial
    (bssmppi_solve_partial); one all-gather of the 3 + 2T partials (NCCL on the device, gloo through
    the host); every rank merges them (bssmppi_merge_partials) into the whole solve's update and
    shifts its resident nominal. A step is that whole solve; value = K M T / the slowest rank's step."""
    import torch

    from paper_2408_00494_gb300 import bssmppi

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    p = _problem(args.workload)
    k0, k1 = rank * p.K // world, (rank + 1) * p.K // world
    q = workload.Problem(**{**p.__dict__, "K": k1 - k0})
    ctl = bssmppi.Controller(q, stream=stream)
    h = ctl.h
    bssmppi.set_sample_range(h, k0, p.K)
    x0 = torch.as_tensor(workload.racing_x0(p), device=dev)
    u0 = torch.zeros(2, device=dev)
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)
    dist = torch.distributed if world > 1 else None

    def step(x):
        bssmppi.sharded_solve(h, x, p.T, u0=u0)
        bssmppi.shift(h, None, 1)

    for _ in range(args.warmup):
        step(x0)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local_rank)
    clocks.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(float(i))
        starts[i].record(stream)
        step(x0)
        ends[i].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    mean_ms = statistics.fmean(s.elapsed_time(e) for s, e in zip(starts, ends))
    # end to end through the binding: H2D of the state from pinned memory, the sharded solve and
    # shift, D2H of u0 into pinned memory, wall clock per step
    x0_h = torch.as_tensor(workload.racing_x0(p)).pin_memory()
    u0_h = torch.zeros(2).pin_memory()
    x0_d = torch.empty(p.nx, device=dev)
    e2e = []
    for i in range(args.warmup + args.steps):
        flush.fill_(float(i))
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        x0_d.copy_(x0_h, non_blocking=True)
        step(x0_d)
        u0_h.copy_(u0, non_blocking=True)
        torch.cuda.synchronize()
        if i >= args.warmup:
            e2e.append(time.perf_counter() - t0)
    ctl.close()
    mean_ms, e2e_ms = reduce_over_ranks([mean_ms, statistics.fmean(e2e) * 1e3], dev, world)
    units = p.K * p.M * p.T
    line = {"metric": METRIC, "value": units / (mean_ms * 1e-3), "unit": "particle-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean_ms, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {**_workload_desc(p, args.workload), "parallelism": f"K split over {world} ranks"},
            "solves_per_s": 1e3 / mean_ms,
            "e2e": {"value": units / (e2e_ms * 1e-3), "unit": "particle-steps/s",
                    "h2d_bytes_per_step": 4 * p.nx, "d2h_bytes_per_step": 8,
                    "exchange_bytes_per_rank": 4 * (3 + 2 * p.T)},
            "gpu_launches": 3 * args.steps,  # per step and rank: partial solve, merge, shift
            "clocks": clk}
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = run_cpu_baseline(p, args.cpu_budget)
    return line


def _relaunch_under_torchrun(args) -> int:
    """--gpus N > 1 without a launcher: run this script as N ranks under torch.distributed.run."""
    import socket

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={args.gpus}",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__), *sys.argv[1:]]
    return subprocess.call(cmd)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", default=None,
                    help="racing_K4096_M64_T40 (default), racing_K256_M16_T20 or racing_K16384_M128_T60 "
                         "(the default of --mode shard)")
    ap.add_argument("--mode", choices=("replicas", "shard"), default="replicas")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--ref-samples", type=int, default=1024)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--closed-loop-steps", type=int, default=1000)
    ap.add_argument("--serve-seconds", type=float, default=1.0)
    ap.add_argument("--serve-sweep-seconds", type=float, default=1.0, help="length of one window of the rate sweep")
    ap.add_argument("--serve-slots", type=int, default=SERVE_SLOTS, help="batches the batched server keeps in flight (1-8)")
    ap.add_argument("--serve-repeats", type=int, default=1, help="windows per rate of the sweep (independent streams)")
    ap.add_argument("--serve-rates", type=lambda s: tuple(float(x) for x in s.split(",")),
                    default=(0.5, 1.0, 1.5, 2.0, 2.5, 3.0, 3.5, 4.0, 4.5, 5.0, 5.5, 6.0, 6.5, 7.0, 7.5),
                    help="per-controller rates of the sweep (Hz)")
    ap.add_argument("--serve-batch-work", type=float, default=SERVE_BATCH_WORK,
                    help="particle-steps admitted per serving batch (bounds a batch's duration)")
    ap.add_argument("--repair-iters", type=int, default=5)
    ap.add_argument("--repair-step", type=float, default=2e-6)
    ap.add_argument("--km-sweep", default="", help="closed-loop lap study over 'K1,K2,...;M1,M2,...' (off by default)")
    ap.add_argument("--km-runs", type=int, default=20)
    ap.add_argument("--km-T", type=int, default=20)
    ap.add_argument("--km-noise", type=float, default=4.0)
    ap.add_argument("--km-speed", type=float, default=10.0)
    ap.add_argument("--km-wT", type=float, default=2.0)
    ap.add_argument("--km-qey", default="0.1", help="lateral-deviation cost weights q_ey to sweep (comma list)")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.workload is None:
        args.workload = "racing_K16384_M128_T60" if args.mode == "shard" else "racing_K4096_M64_T40"
    if args.gpus < 1:
        raise SystemExit("--gpus must be >= 1")

    if "WORLD_SIZE" not in os.environ and args.gpus > 1:
        raise SystemExit(_relaunch_under_torchrun(args))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world != args.gpus:
        raise SystemExit(f"--gpus {args.gpus} but the launcher started {world} ranks (WORLD_SIZE)")

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return

    if world > 1:
        import torch
        torch.distributed.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")
    try:
        line = (run_shard if args.mode == "shard" else run_ours)(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
