#!/usr/bin/env python
"""Benchmark of the SMC-MPC hot path on GB300.

One step = one SMC solve (Algorithm 1) of the high-density TMA workload
(24 aircraft, L = 262144 particles, M = 64 wind samples, H = 120 steps,
64x64x8 wind grid, 30 annealing iterations, fuel + ground-noise cost, hard and
softplus separation both evaluated): wind-field generation, 30 rollouts with
costs, 29 x (FP64 LSE, systematic resampling, move), final selection.
`--workload c2` times the 8-aircraft workload instead (L = 65536, M = 32,
H = 60, fuel cost, hard separation).
Metric: aircraft-step-samples per second = L*M*N*H*J_max per solve / time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload c3|c2]

Under torchrun (N > 1) every rank solves an independent replica (its own
seed): scaling is weak, no collective touches the data path; the time is the
maximum over ranks.  `--impl reference` times the FP64 CPU oracle on the host
cores (rank 0 only) on a bounded sample of the same workload.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "aircraft-step-samples/sec"
UNIT = "aircraft-step-samples/s"
# The timed workloads: the scenario generator, the name the line reports, and
# the oracle's sample sizes (particles) for the CPU baseline, the reference arm
# and the rollout-only rates (single-threaded, all cores).
WORKLOADS = {
    "c3": dict(config=3, name="tma-24ac-L262144-M64-H120-grid64x64x8-J30-noise-hardsoft",
               cpu_particles=64, reference_particles=32, rollout_one=32, rollout_all=512),
    "c2": dict(config=2, name="tma-8ac-L65536-M32-H60-grid64x64x8-J30",
               cpu_particles=512, reference_particles=256, rollout_one=256, rollout_all=4096),
}

# Peaks: measured copy bandwidth from MEASURED_PEAKS.json when present; the FP32
# CUDA-core peak is derived: SMs x 128 FP32 lanes x 2 flop/FMA x SM clock, with
# the SM count from the device and the clock sampled during the timed region.
FP32_LANES = 128


def fp32_peak_tflops(sms, sm_mhz):
    return sms * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12


def flops_per_unit(p, particles=8, samples=2):
    """Algorithmic floating-point operations per live aircraft-step-sample (one
    aircraft advanced one step under one wind sample in one particle), counted
    mechanically on the FP64 oracle's rollout (the operation-counting build of
    oracle/opcount.cpp: +, -, *, /, comparisons, min/max/abs and each
    elementary function 1; an FMA is two of them) of `particles` uniform
    initial particles under the first `samples` wind samples of the workload,
    costs included (the soft form too when the solve computes it); pairs are
    checked once per unordered pair, as in the oracle."""
    import oracle as O
    q = p.copy(L=particles, M=samples)
    W = O.wind_field(q)
    u = O.init_controls(q, particles)
    ops, live = O.rollout_opcount(q, u, 0, W, soft=(q.sep_mode != 0))
    return ops / live


def flops_per_unit_isolated(workload):
    """flops_per_unit of the named workload, counted in a child process (the
    counting build of the oracle never shares a process with the timed GPU
    work); None if the child fails."""
    code = ("import sys; sys.path.insert(0, %r); import bench; "
            "print(bench.flops_per_unit(bench.workload_problem(%r)))" % (ROOT, workload))
    try:
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
        return float(r.stdout.strip().splitlines()[-1]) if r.returncode == 0 else None
    except (OSError, ValueError, IndexError, subprocess.SubprocessError):
        return None


def flops_per_unit_tally(p):
    """The same work tallied by hand from the per-step formulas (for
    comparison): +, -, *, /, sqrt, min/max/compare and each elementary function
    count 1, an FMA 2.  Pairwise separation is counted once per unordered pair
    ((N-1)/2 pairs per unit)."""
    import numpy as np
    base = 31 + 1        # control-derived quantities, limits, mass
    wind = 21 + 28       # cell search in 3 axes, 7 lerps x 2 components
    turb = 8 + 4         # Box-Muller per 2 normals (2 per step), 2 fma
    euler = 24           # sincos, position/altitude/speed/heading, fuel (Kahan), unary checks
    arr = 38             # bearing, arc, glide angle, landing sector, two compensated sums
    dep = 22             # bearing error, altitude and speed deviations, three compensated sums
    noise = 14 if p.w_noise != 0 else 0
    pair = 8 + (9 if p.sep_mode != 0 else 0)
    frac_arr = float(np.mean(p.aircraft["type"] == 0))
    return base + wind + turb + euler + frac_arr * arr + (1 - frac_arr) * dep + noise + \
        pair * (p.N - 1) / 2.0


# DRAM bytes (read + write) of one full-size rollout launch per workload and
# rollout kernel, from a one-pass ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum of one launch late in a solve: iteration 20 of 30);
# valid only for the kernel sources they were taken on.
ROLLOUT_TRAFFIC = {"sources_sha256_16": "9c6681ad7c36f584",
                   "bytes_per_launch": {"c3:rollout_kernel": 47479898368 + 4464612352}}


def rollout_kernel_name(variant):
    """The rollout kernel a launch variant runs (8-12: two wind samples per thread; 13-15 and
    16-17 the one-sample kernel on 16- and 8-particle tiles)."""
    return "rollout_pair_kernel" if variant is not None and 8 <= variant < 13 else "rollout_kernel"


def rollout_sources_digest():
    h = hashlib.sha256()
    for f in ("rollout.cu", "rollout_pair.cu", "rollout_tile.cuh", "device_common.cuh"):
        with open(os.path.join(ROOT, "paper_1506_02869_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clock / throttle samples of one GPU during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.uuid, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for name, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value, world, device=None):
    """Maximum of a float over all ranks (the slowest rank sets the time)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload_problem(workload, seed=None):
    import scenarios as S
    cfg = WORKLOADS[workload]["config"]
    return S.make_config(cfg) if seed is None else S.make_config(cfg, seed=seed)


def replica_problem(rank, workload="c3", base_seed=None):
    """Rank r solves an independent replica of the workload with its own seed."""
    p = workload_problem(workload, base_seed)
    return p.copy(seed=p.seed + 1000003 * rank)


def units_per_solve(p):
    return p.L * p.M * p.N * p.H * p.J_max


# ----------------------------------------------------------------- CPU oracle

_ORACLE_WIND = {}


def oracle_wind(workload):
    """The workload's wind field from the oracle (FP64), generated once per
    process; returns (field, generation seconds)."""
    import oracle as O
    if workload not in _ORACLE_WIND:
        t0 = time.perf_counter()
        W = O.wind_field(workload_problem(workload))
        _ORACLE_WIND[workload] = dict(W=W, seconds=time.perf_counter() - t0)
    return _ORACLE_WIND[workload]["W"], _ORACLE_WIND[workload]["seconds"]


def oracle_sample(workload, L_sample, nthreads):
    """The FP64 oracle's full solve on the workload's traffic with L_sample
    particles (all other sizes full) on the workload's wind field, whose
    generation time is charged at the share L_sample / L of the full
    workload's (the field does not depend on L; a solve of L_sample particles
    that generated it again would carry all of it); returns (units/s,
    seconds, units)."""
    import oracle as O
    W, t_wind = oracle_wind(workload)
    full = workload_problem(workload)
    p = full.copy(L=L_sample)
    t0 = time.perf_counter()
    O.smc_solve(p, W=W, nthreads=nthreads)
    dt = time.perf_counter() - t0 + t_wind * L_sample / full.L
    u = units_per_solve(p)
    return u / dt, dt, u


def oracle_rollout_rates(workload, L_one, L_all, cores):
    """The oracle's rollout alone (one iteration's inner loop on the uniform
    initial controls, the workload's wind field computed beforehand), single-
    threaded on L_one particles and on all cores on L_all; returns
    {threads: (units/s, seconds, units, particles)} with units = L M N H."""
    import oracle as O
    p = workload_problem(workload)
    W, _ = oracle_wind(workload)
    out = {}
    for L, n in ((L_one, 1), (L_all, cores)) if cores > 1 else ((L_one, 1),):
        q = p.copy(L=L)
        u = O.init_controls(q, L)
        t0 = time.perf_counter()
        O.rollout(q, u, 0, W=W, nthreads=n, soft=(q.sep_mode != 0))
        dt = time.perf_counter() - t0
        units = L * q.M * q.N * q.H
        out[n] = (units / dt, dt, units, L)
    return out


def cpu_model():
    """The host CPU's model name (lscpu), else the machine type."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            key, _, val = line.partition(":")
            if key.strip() == "Model name" and val.strip():
                return val.strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.processor() or platform.machine()


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    cores = os.cpu_count() or 1
    wl = WORKLOADS[args.workload]
    Ls = args.reference_particles or wl["reference_particles"]
    for _ in range(args.warmup):
        oracle_sample(args.workload, Ls, cores)
    times, units = [], 0
    for _ in range(args.steps):
        _, dt, units = oracle_sample(args.workload, Ls, cores)
        times.append(dt)
    tot = sum(times)
    value = units * args.steps / tot
    _, t_wind = oracle_wind(args.workload)
    full = workload_problem(args.workload)
    sample = (f"oracle smc_solve of the workload's traffic with L={Ls} particles "
              f"(M={full.M}, N={full.N}, H={full.H}, J_max={full.J_max}) on the "
              f"{'x'.join(str(g) for g in full.grid)} wind field, whose generation "
              f"({t_wind:.1f} s, once) is charged at the share {Ls}/{full.L} per step; {cores} threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl["name"], "sample_particles": Ls, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm

def run_ours(args, world, rank, local):
    import ctypes as C

    import numpy as np
    import torch

    import paper_1506_02869_gb300 as pkg

    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=device)
    pkg.build()
    lib = pkg.lib()
    wl = WORKLOADS[args.workload]
    p = replica_problem(rank, args.workload)
    solver = pkg.Solver(p, device=device)
    h = solver.h
    stream = torch.cuda.current_stream(device)
    best_u = torch.empty((p.N, p.S, 3), dtype=torch.float32, device=device)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier(device_ids=[local])

    # warm-up (also builds the wind-covariance factors)
    for _ in range(args.warmup):
        pkg.tma_solve(h, best_u, want_cost=False)
    torch.cuda.synchronize(device)

    # ---- timed region: K solves with inputs resident on the device
    pkg.tma_profile_enable(h, True)
    pkg.tma_profile_read(h, reset=True)
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(device).uuid)
    except Exception:
        pass
    sampler = ClockSampler(uuid) if uuid else None
    barrier()
    torch.cuda.synchronize(device)
    if sampler:
        sampler.start()
        time.sleep(0.3)
    n0 = lib.tma_launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        pkg.tma_solve(h, best_u, want_cost=False)
    ev1.record(stream)
    torch.cuda.synchronize(device)
    launches = lib.tma_launch_count() - n0
    clocks = sampler.stop() if sampler else None
    barrier()
    elapsed_ms = ev0.elapsed_time(ev1)
    prof = pkg.tma_profile_read(h, reset=True)
    pkg.tma_profile_enable(h, False)
    live_per_solve = pkg.tma_live_steps(h)
    elapsed_max = max_over_ranks(elapsed_ms, world, device)
    units = units_per_solve(p)
    value = units * args.steps * world / (elapsed_max * 1e-3)

    # ---- end to end: host state in, host controls out, through the C-ABI (the
    # same solve, at most --e2e-steps of them when the device-timed loop is longer)
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    x0 = torch.tensor([[float(a[k]) for k in ("x", "y", "z", "v", "chi", "m")] for a in p.aircraft],
                      dtype=torch.float64).pin_memory()
    out_h = torch.empty((p.N, p.S, 3), dtype=torch.float32).pin_memory()
    cost = C.c_double()
    statuses = set()
    barrier()
    torch.cuda.synchronize(device)
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        st = lib.tma_solve_host(h, C.cast(C.c_void_p(x0.data_ptr()), C.POINTER(pkg.TmaState)),
                                p.mpc_step, C.c_void_p(out_h.data_ptr()), C.byref(cost),
                                pkg._stream(stream))
        statuses.add(st)
    torch.cuda.synchronize(device)
    e2e_s = time.perf_counter() - t0
    barrier()
    e2e_max = max_over_ranks(e2e_s, world, device)
    if statuses - {pkg.TMA_OK, pkg.TMA_WARN_DEGENERATE}:
        raise RuntimeError(f"tma_solve_host failed: {statuses}")
    e2e_value = units * e2e_steps * world / e2e_max

    # ---- roofline of the rollout kernel (the dominant kernel)
    roll_ms, roll_n = prof["rollout"]
    fpu_counted = flops_per_unit_isolated(args.workload)
    fpu = fpu_counted if fpu_counted else flops_per_unit_tally(p)
    live_per_launch = live_per_solve / p.J_max
    achieved = fpu * live_per_launch / (roll_ms / roll_n * 1e-3) / 1e12 if roll_n else None
    # FP32 peak at the SM clock sampled during the timed region (else the
    # measured maximum clock), on the device's SM count
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    pk = measured_peaks()
    if clocks and clocks.get("sm_mhz"):
        sm_clock, clock_src = float(clocks["sm_mhz"]), "median SM clock sampled during the timed region"
    elif pk and pk.get("sm_max_mhz"):
        sm_clock, clock_src = float(pk["sm_max_mhz"]), "maximum SM clock of MEASURED_PEAKS.json"
    else:
        sm_clock, clock_src = 2070.0, "nominal maximum SM clock"
    peak = fp32_peak_tflops(sms, sm_clock)
    total_ms = sum(v[0] for v in prof.values())
    variant, timed = pkg.tma_get_tuning(h)
    kname = rollout_kernel_name(variant)
    roofline = {
        "bound": "alu", "kernel": kname, "achieved": achieved, "peak": peak,
        "unit": "TFLOP/s", "frac": (achieved / peak) if achieved else None,
        "traffic": (ROLLOUT_TRAFFIC["bytes_per_launch"].get(f"{args.workload}:{kname}")
                    if rollout_sources_digest() == ROLLOUT_TRAFFIC["sources_sha256_16"] else None),
        "peak_source": f"derived: {sms} SMs x {FP32_LANES} FP32 lanes x 2 flop x {sm_clock:.0f} MHz "
                       f"({clock_src})",
        "flops_per_unit": fpu,
        "flops_per_unit_source": ("counted on the FP64 oracle's rollout (oracle/opcount.cpp), 8 uniform "
                                  "initial particles x 2 wind samples" if fpu_counted else
                                  "hand tally (the counting run failed)"),
        "flops_per_unit_hand_tally": flops_per_unit_tally(p), "live_units_per_launch": live_per_launch,
        "units_per_launch": p.L * p.M * p.N * p.H, "launch_ms": roll_ms / roll_n if roll_n else None,
        "stage_ms_share": {k: round(v[0] / total_ms, 4) for k, v in prof.items() if total_ms},
    }
    if pk:
        roofline["hbm_peak_gbs_measured"] = pk.get("hbm_gbs")
    roofline["launch_variant"] = {"chosen": variant,
                                  "timed_ms": {str(k): round(v, 4) for k, v in timed.items()}}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": wl["name"], "L": p.L, "M": p.M, "N": p.N, "H": p.H, "J_max": p.J_max,
                   "grid": list(p.grid), "noise_weight": p.w_noise, "sep_mode": p.sep_mode,
                   "parallelism": f"replicas{world}", "e2e_steps": e2e_steps,
                   "l2": f"inputs larger than L2 (packed wind field "
                         f"{p.M * p.H * p.n_grid * 16 / 1e9:.1f} GB per solve)"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(x0.numel() * 8),
                "d2h_bytes_per_step": int(out_h.numel() * 4 + 8 + 4)},
        "gpu_launches": int(launches),
        "roofline": roofline,
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        Lc = args.cpu_particles or wl["cpu_particles"]
        v, dt, u = oracle_sample(args.workload, Lc, cores)
        line["cpu_baseline"] = {
            "value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"one oracle smc_solve of the workload's traffic with L={Lc} "
                       f"particles (full M, N, H, J_max) on the wind field, whose generation "
                       f"({oracle_wind(args.workload)[1]:.1f} s) is charged at the share {Lc}/{p.L}: "
                       f"{u:.3g} units in {dt:.1f} s"),
            "cpu_model": cpu_model()}
        rr = oracle_rollout_rates(args.workload, wl["rollout_one"], wl["rollout_all"], cores)
        line["cpu_baseline"]["rollout_only"] = {
            f"threads_{n}": {"value": v_, "unit": UNIT,
                             "sample": f"one oracle rollout (J = 0, initial controls, wind precomputed) of "
                                       f"L={L_} particles: {u_:.3g} units in {dt_:.2f} s"}
            for n, (v_, dt_, u_, L_) in rr.items()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    solver.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_rollout_only(args, local):
    """Small rollout-only case for kernel profiling: the workload's traffic and
    wind field with `--particles` particles, uniform initial controls, K rollouts."""
    import torch

    import paper_1506_02869_gb300 as pkg
    import scenarios as S

    torch.cuda.set_device(local)
    pkg.build()
    p = S.make_config(args.config).copy(L=args.particles or 4096)
    if args.samples:
        p = p.copy(M=args.samples)
    if args.wind != "shared":
        # the 2x2x2 grid of the box corners: one shared field, or one per particle
        p = p.copy(grid=(2, 2, 2), wind_mode=1 if args.wind == "own" else 0)
    solver = pkg.Solver(p)
    if args.late:
        # the particles of a finished solve: the live mix of the late iterations
        solver.solve()
        u = solver.particles()
        J0 = p.J_max - 1
    else:
        u = solver.init_controls()
        J0 = 0
    soft = p.sep_mode != 0        # the solve's rollout computes the soft costs too
    for _ in range(args.warmup):
        solver.rollout_cost(u, J0, soft=soft)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for j in range(args.steps):
        solver.rollout_cost(u, J0, soft=soft)
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / max(args.steps, 1)
    units = p.L * p.M * p.N * p.H
    print(json.dumps({"mode": "rollout-only", "config": args.config, "N": p.N, "late": bool(args.late),
                      "wind": args.wind,
                      "particles": p.L, "ms_per_rollout": ms,
                      "units_per_s": units / (ms * 1e-3), "live_steps": solver.live_steps()}))
    solver.close()
    return 0


def run_grad_only(args, local):
    """Small gradient-only case for kernel profiling: the softplus-separation
    workload (12 aircraft, M 16, H 60) with `--particles` particles, uniform
    controls, K gradient passes."""
    import torch

    import paper_1506_02869_gb300 as pkg
    import scenarios as S

    torch.cuda.set_device(local)
    pkg.build()
    p = S.config4().copy(L=args.particles or 4096)
    solver = pkg.Solver(p)
    if args.late:
        solver.solve()
        u = solver.particles()
        J0 = p.J_max - 1
    else:
        u = solver.init_controls()
        J0 = 0
    for _ in range(args.warmup):
        solver.rollout_grad(u, J0)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for j in range(args.steps):
        solver.rollout_grad(u, J0)
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / max(args.steps, 1)
    units = p.L * p.M * p.N * p.H
    print(json.dumps({"mode": "grad-only", "late": bool(args.late), "particles": p.L, "ms_per_gradient": ms,
                      "units_per_s": units / (ms * 1e-3),
                      "grad_tuning": pkg.tma_get_grad_tuning(solver.h)}))
    solver.close()
    return 0


def run_stages(args, local):
    """The HBM-side stages between rollouts on the 24-aircraft workload (L 262144):
    FP64 log-weight normalisation, systematic resampling and gather + move, each
    timed alone with CUDA events (20 back-to-back calls per step, median over K
    steps; inputs larger than L2).
    Algorithmic bytes per (aircraft, particle): normalisation 4 B read + 8 B
    written; resampling 8 B read + 4 B written; move 4 B ancestor + 48 B parent +
    48 B child."""
    import numpy as np
    import torch

    import paper_1506_02869_gb300 as pkg
    import scenarios as S

    torch.cuda.set_device(local)
    pkg.build()
    p = S.config3()
    N, L = p.N, p.L
    g = torch.Generator(device="cuda").manual_seed(7)
    cbar = (2.0 * torch.rand((N, L), device="cuda", generator=g)).float()
    cbar[torch.rand((N, L), device="cuda", generator=g) < 0.05] = float("inf")
    wt = torch.empty((N, L), dtype=torch.float64, device="cuda")
    anc = torch.empty((N, L), dtype=torch.int32, device="cuda")
    only = args.stage
    # the move's solver (the workload's wind field, several GB) only when the move is timed
    sol = pkg.Solver(p) if only in ("all", "move") else None
    u = sol.init_controls() if sol else None
    u2 = torch.empty_like(u) if sol else None
    lwork = torch.empty(pkg.lib().tma_lse_workspace(N, L), dtype=torch.uint8, device="cuda")
    rwork = torch.empty(pkg.lib().tma_resample_workspace(N, L), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def med_ms(fn, reps=20):
        # back-to-back calls between the events, so that host-side call overhead
        # overlaps device work; median over the steps of the per-call time
        for _ in range(args.warmup):
            fn()
        ts = []
        for _ in range(max(args.steps, 1)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) / reps)
        return float(np.median(ts))

    fwork = torch.empty(pkg.lib().tma_lse_resample_workspace(N, L), dtype=torch.uint8, device="cuda")
    deg = torch.zeros(1, dtype=torch.int32, device="cuda")
    kappa = 11.0
    calls = {
        "lse": lambda: pkg.tma_lse(cbar, kappa, wt, work=lwork),
        "resample": lambda: pkg.tma_resample(wt, p.seed, 0, 3, 0, anc, work=rwork),
        "lse_resample": lambda: pkg.tma_lse_resample(cbar, kappa, p.seed, 0, 3, 0, wt, anc, deg, work=fwork),
        "move": lambda: pkg.tma_move(sol.h, u, anc, 3, u2),
    }
    if only != "all" and only != "lse":
        pkg.tma_lse(cbar, kappa, wt, work=lwork)         # weights for the resampling on its own
    if only == "move":
        pkg.tma_resample(wt, p.seed, 0, 3, 0, anc, work=rwork)   # the move's ancestors
    ms = {k: med_ms(f) for k, f in calls.items() if only in ("all", k)}
    if sol:
        sol.close()
    peaks = measured_peaks() or {}
    hbm = peaks.get("hbm_gbs") or 6800.0
    hbm_source = "measured" if peaks.get("hbm_gbs") else "fallback"
    n = N * L
    # the fused call reads the costs, writes and reads wtilde once each, writes
    # the ancestors; "resample" alone (tma_resample) also synchronises the
    # stream to read its degenerate status, so its time includes that round trip
    algo = {"lse": 12, "resample": 12, "lse_resample": 24, "move": 100}
    out = {"mode": "stages", "workload": "tma-24ac-L262144 (nseg 24)", "elements": n,
           "hbm_peak_gbs": hbm, "hbm_peak_source": hbm_source, "stages": {}}
    for k, v in ms.items():
        gbs = algo[k] * n / (v * 1e-3) / 1e9
        out["stages"][k] = {"ms": round(v, 4), "algorithmic_bytes_per_element": algo[k],
                            "achieved_gbs": round(gbs, 1), "frac_of_hbm_peak": round(gbs / hbm, 3)}
    # the normalisation evaluates one FP64 exp per element
    if "lse" in ms:
        out["stages"]["lse"]["fp64_exp_per_s"] = round(n / (ms["lse"] * 1e-3), 1)
    # the resampling's share of the fused call (its expansion pass: wtilde read,
    # ancestors written), by difference from the normalisation alone
    d = ms["lse_resample"] - ms["lse"] if "lse" in ms and "lse_resample" in ms else 0.0
    if d > 0:
        gbs = 12 * n / (d * 1e-3) / 1e9
        out["stages"]["resample_in_fused_call"] = {"ms": round(d, 4), "algorithmic_bytes_per_element": 12,
                                                   "achieved_gbs": round(gbs, 1),
                                                   "frac_of_hbm_peak": round(gbs / hbm, 3)}
    print(json.dumps(out), flush=True)
    return 0


def run_batched(args, local):
    """Batched MPC workload: n scenarios with N_s ~ U{2..32}, L 16384, M 16,
    H 60, J_max 20, 16x16x4 wind grid; one step = --mpc-steps receding-horizon
    steps of all scenarios (solve + plant), captured as one CUDA graph (the
    time includes the capture, a fraction of a second).  Beside it, the plain
    form on the same GPU: one solver per scenario, solved one after the other
    (solve + plant step per MPC step), on a sample of --single-sample
    scenarios spread over the aircraft counts (throughput is per unit of
    work)."""
    import numpy as np
    import torch

    import paper_1506_02869_gb300 as pkg
    import scenarios as S

    torch.cuda.set_device(local)
    pkg.build()
    ps = S.config5(n_scen=args.scenarios)
    if args.particles:
        ps = [S.shrink(p, L=args.particles) for p in ps]
    Ns = [p.N for p in ps]
    t0 = time.perf_counter()
    b = pkg.tma_batch_create(ps)
    create_s = time.perf_counter() - t0
    form, timed = pkg.tma_batch_get_dispatch(b)
    units = sum(p.L * p.M * p.N * p.H * p.J_max for p in ps) * args.mpc_steps
    stream = torch.cuda.current_stream()
    out = {"mode": "batched", "scenarios": len(ps), "aircraft": int(sum(Ns)),
           "mpc_steps_per_step": args.mpc_steps, "L": ps[0].L, "M": ps[0].M, "H": ps[0].H,
           "J_max": ps[0].J_max, "metric": METRIC, "unit": UNIT,
           "dispatch": {"chosen": ["persistent launch", "launch per scenario"][form],
                        "rollout_ms_persistent": timed[0], "rollout_ms_per_scenario": timed[1],
                        "create_s": round(create_s, 2)}}
    for _ in range(args.warmup):
        pkg.tma_batch_mpc(b, args.mpc_steps, use_graph=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lat = []
    ms_total = 0.0
    for _ in range(args.steps):
        e0.record(stream)
        pkg.tma_batch_mpc(b, args.mpc_steps, use_graph=True)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_total += e0.elapsed_time(e1)
        lat.append(pkg.tma_batch_latency(b, len(ps)))
    lat = np.concatenate(lat)
    out["graph"] = {"value": units * args.steps / (ms_total * 1e-3), "ms_per_step": ms_total / args.steps,
                    "ms_per_mpc_step": ms_total / args.steps / args.mpc_steps,
                    "solve_latency_ms_p50": float(np.percentile(lat, 50)),
                    "solve_latency_ms_p99": float(np.percentile(lat, 99)),
                    "latency_note": "every scenario's selection is in the same final stage of the solve "
                                    "(the stages run over all scenarios together), so all scenarios "
                                    "finish together: p50 = p99 by construction"}
    out["live_steps_last_solve"] = pkg.tma_batch_live_steps(b)
    pkg.tma_batch_destroy(b)
    # the plain form: one solver per scenario of a sample spread over the counts
    order = sorted(range(len(ps)), key=lambda k: Ns[k])
    n_s = max(1, min(args.single_sample, len(ps)))
    pick = [order[int(round(q))] for q in np.linspace(0, len(ps) - 1, n_s)]
    sols = [pkg.Solver(ps[k]) for k in pick]
    for sol in sols[:2]:
        sol.solve()
    torch.cuda.synchronize()
    lat = []
    ms_total = 0.0
    for _ in range(args.mpc_steps):
        for sol in sols:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            bu, _, _ = sol.solve()
            pkg.tma_plant_step(sol.h, bu)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            ms_total += ms
            lat.append(ms)
    for sol in sols:
        sol.close()
    units_s = sum(ps[k].L * ps[k].M * ps[k].N * ps[k].H * ps[k].J_max for k in pick) * args.mpc_steps
    out["single"] = {"scenarios": n_s, "aircraft": int(sum(Ns[k] for k in pick)),
                     "value": units_s / (ms_total * 1e-3), "ms_total": ms_total,
                     "solve_latency_ms_p50": float(np.percentile(lat, 50)),
                     "solve_latency_ms_p99": float(np.percentile(lat, 99))}
    out["batched_over_single"] = out["graph"]["value"] / out["single"]["value"]
    print(json.dumps(out), flush=True)
    return 0


def run_moves(args, local):
    """Moves between the SMC iterations on the softplus-separation workload
    (12 aircraft, L 16384, M 16, H 60, 16x16x4 wind grid): the paper's clipped
    random walk, a random walk with a Metropolis-Hastings accept step, and the
    Langevin proposal with accept step.  For every seed (a new traffic scenario
    and random streams) each kind solves with J_max on a ladder; the chosen
    controls are scored on 256 held-out wind samples (random stream 8) as
    sum_i cbar_soft[i].  Target: the paper move's held-out cost at the full
    J_max.  Time to target = device time of the first ladder solve whose
    held-out cost is at most the target."""
    import numpy as np
    import torch

    import paper_1506_02869_gb300 as pkg
    import scenarios as S

    torch.cuda.set_device(local)
    pkg.build()
    base = S.config4()
    ladder = [j for j in (2, 4, 6, 8, 12, 16, 20, 25, 30) if j <= base.J_max]
    kinds = {0: ("paper", None), 1: ("rw_mh", args.eps_rw), 2: ("mala", args.eps_mala)}
    n_seeds = args.seeds
    stream = torch.cuda.current_stream()

    def timed_solve(p, kind):
        sol = pkg.Solver(p)
        if kind:
            sol.set_move(kind, kinds[kind][1])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        bu, _, _ = sol.solve()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        acc = sol.mh_stats()[0] / p.L if kind else None
        sol.close()
        return bu, ms, acc

    # warm-up (module load, autotuning, allocation paths)
    for k in kinds:
        timed_solve(base.copy(J_max=2), k)

    res = {kinds[k][0]: {"heldout": [], "ms": []} for k in kinds}
    acc_example = {}
    for s in range(n_seeds):
        p = S.config4(seed=base.seed + 1000 * s)
        ev = pkg.Solver(p.copy(M=256, L=32))
        ev.set_wind_stream(8)
        ev.wind_field()
        for k, (name, _) in kinds.items():
            hs, ts = [], []
            for J in ladder:
                bu, ms, acc = timed_solve(p.copy(J_max=J), k)
                _, cs = ev.rollout_cost(bu[None].contiguous(), 0, soft=True)
                hs.append(float(cs[:, 0].double().sum().item()))
                ts.append(ms)
                if s == 0 and J == ladder[-1] and acc is not None:
                    acc_example[name] = [round(float(a), 3) for a in acc]
            res[name]["heldout"].append(hs)
            res[name]["ms"].append(ts)
        ev.close()
    out = {"mode": "moves", "workload": "tma-12ac-L16384-M16-H60-grid16x16x4-softplus",
           "seeds": n_seeds, "ladder_J_max": ladder, "heldout_samples": 256,
           "eps0": {"rw_mh": args.eps_rw, "mala": args.eps_mala},
           "acceptance_per_iteration_seed0": acc_example}
    # one rollout and one gradient pass on the full workload (J = 3)
    sol = pkg.Solver(base)
    u = sol.init_controls()
    sol.rollout_grad(u, 3)
    cb = torch.empty((base.N, base.L), device="cuda")

    def med_ms(fn, reps=5):
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    ms_roll = med_ms(lambda: pkg.tma_rollout_cost(sol.h, u, 3, cb, torch.empty_like(cb)))
    ms_grad = med_ms(lambda: sol.rollout_grad(u, 3))
    gv, gt = pkg.tma_get_grad_tuning(sol.h)
    sol.close()
    out["full_workload_ms"] = {"rollout_soft": round(ms_roll, 3), "gradient": round(ms_grad, 3),
                               "gradient_over_rollout": round(ms_grad / ms_roll, 2),
                               "grad_variant": gv,
                               "grad_variants_timed_ms": {str(k): round(v, 3) for k, v in gt.items()}}
    target = np.array([h[-1] for h in res["paper"]["heldout"]])
    for name, r in res.items():
        H = np.array(r["heldout"])
        T = np.array(r["ms"])
        ttt = []
        for s in range(n_seeds):
            hit = np.nonzero(H[s] <= target[s])[0]
            ttt.append(float(T[s, hit[0]]) if hit.size else float("inf"))
        ttt = np.array(ttt)
        out[name] = {
            "median_time_to_target_ms": float(np.median(ttt)),
            "reached": int(np.isfinite(ttt).sum()),
            "median_heldout_cost_at_full_J": float(np.median(H[:, -1])),
            "median_heldout_cost_per_rung": [round(float(v), 4) for v in np.median(H, axis=0)],
            "median_solve_ms_per_rung": [round(float(v), 2) for v in np.median(T, axis=0)],
        }
    print(json.dumps(out), flush=True)
    return 0


def run_schedule(args, local):
    """Fixed against scheduled work on the headline workload (config 2:
    L 65536, N 8, H 60, 64x64x8 grid, J_max 30; M = 32 samples allocated).
      fixed:     every iteration rolls out all 32 samples of all 65536 particles
                 (exponent kappa_J);
      samples:   sample mode 1, the inner loop of Algorithm 1 (iteration J rolls
                 out min(SampleSchedule(J), 32) samples, weight = their product);
      particles: a particle count falling geometrically from 65536 to 8192
                 (the speed-up the paper proposes), all 32 samples;
      both:      the two schedules together.
    Per seed (new traffic and streams) every variant solves; the chosen controls
    are scored on 256 held-out wind samples (random stream 8) as sum_i cbar[i]."""
    import numpy as np
    import torch

    import paper_1506_02869_gb300 as pkg
    import scenarios as S

    torch.cuda.set_device(local)
    pkg.build()
    base = S.config2()
    stream = torch.cuda.current_stream()
    lsched = S.particle_schedule(base.L, base.J_max, 0.125)
    variants = {"fixed": {}, "samples": {"sample_mode": 1}, "particles": {"L_sched": lsched},
                "both": {"sample_mode": 1, "L_sched": lsched}}

    def samples_of(p, J):
        k = int(np.floor(3.0 + 5.0 * np.exp(0.05 * J)))
        return min(k, p.M) if p.sample_mode == 1 else p.M

    def particles_of(p, J):
        return p.L_sched[J] if p.L_sched is not None else p.L

    tuned = {}

    def timed_solve(p):
        sol = pkg.Solver(p)
        tuned[p.N] = pkg.tma_get_tuning(sol.h)[0]
        sol.solve()                       # warm (autotuning, allocation)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        bu, c, _ = sol.solve()
        e1.record(stream)
        torch.cuda.synchronize()
        sol.close()
        return bu, c, e0.elapsed_time(e1)

    res = {m: {"ms": [], "heldout": [], "units": []} for m in variants}
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except (AttributeError, RuntimeError):
        uuid = None
    sampler = ClockSampler(uuid) if uuid else None
    if sampler:
        sampler.start()
    for s in range(args.seeds):
        p0 = S.config2(seed=base.seed + 1000 * s)
        ev = pkg.Solver(p0.copy(M=256, L=32))
        ev.set_wind_stream(8)
        ev.wind_field()
        torch.cuda.synchronize()
        for name, kw in variants.items():
            p = p0.copy(**kw)
            bu, c, ms = timed_solve(p)
            cb, _ = ev.rollout_cost(bu[None].contiguous(), 0)
            res[name]["ms"].append(ms)
            res[name]["heldout"].append(float(cb[:, 0].double().sum().item()))
            res[name]["units"].append(p.N * p.H * sum(samples_of(p, J) * particles_of(p, J)
                                                      for J in range(p.J_max)))
        ev.close()
    out = {"mode": "schedule", "workload": "tma-8ac-L65536-M32-H60-grid64x64x8-J30",
           "seeds": args.seeds, "heldout_samples": 256,
           "samples_per_iteration": [samples_of(base.copy(sample_mode=1), J) for J in range(base.J_max)],
           "particles_per_iteration": list(lsched),
           "clocks": sampler.stop() if sampler else None, "rollout_variant": tuned}
    for name, r in res.items():
        ms = np.array(r["ms"])
        H = np.array(r["heldout"])
        out[name] = {"median_solve_ms": float(np.median(ms)),
                     "work_fraction": round(r["units"][0] / res["fixed"]["units"][0], 4),
                     "aircraft_step_samples_per_s": float(np.median(np.array(r["units"]) / (ms * 1e-3))),
                     "median_heldout_cost": float(np.median(H)),
                     "heldout_cost_per_seed": [round(float(v), 4) for v in H],
                     "feasible": int(np.isfinite(H).sum())}
    print(json.dumps(out), flush=True)
    return 0


def run_layout_sweep(args, local):
    """The paper's layout sweep (Sec. 4.4, Table comp_sense) re-run on GB300 on
    the paper's standard problem: 10 aircraft that all enter the problem at MPC
    step 5 with a horizon of 6 steps (rolling window: partly active horizons
    before that), 10240 particles, J_max = 100 iterations whose inner loop draws
    SampleSchedule(J) = floor(3 + 5 exp(0.05 J)) wind realisations (sample mode
    1, at most 708), each particle's wind on the 2x2x2 grid of the box corners
    drawn inside the kernel (wind mode 1; Sec. 5.1); the time of one MPC update
    (solve + plant step) averaged over the steps after the settling period.
    On GB300 the block is fixed by the mapping (32 particles x N aircraft); what
    varies is the launch-bound variant (block-size cap x minimum resident
    blocks, i.e. registers per thread against resident blocks per SM), each
    forced in turn.  Traffic: the first 10 aircraft of the 12-aircraft
    workload.  The paper's times (GTX 580) are printed beside as context."""
    import numpy as np
    import torch

    import paper_1506_02869_gb300 as pkg
    import scenarios as S

    torch.cuda.set_device(local)
    pkg.build()
    base = S.config4()
    ac = base.aircraft[:10].copy()
    ac["t_enter"] = 5
    p = base.copy(N=10, aircraft=ac, L=10240, H=6, rolling=1, mpc_step=0, J_max=100, sample_mode=1,
                  M=708, wind_mode=1, grid=(2, 2, 2))
    draws = sum(min(math.floor(3 + 5 * math.exp(0.05 * J)), p.M) for J in range(p.J_max))
    units_settled = p.L * draws * p.N * p.H        # every aircraft active over the whole horizon
    names = {0: "256x4", 1: "256x3", 2: "512x2", 3: "512x1", 4: "1024x1", 5: "256x2",
             6: "384x2", 7: "768x1", 8: "pair 256x3", 9: "pair 256x2", 10: "pair 384x2",
             11: "pair 512x1", 12: "pair 768x1"}
    regs = {0: 64, 1: 85, 2: 64, 3: 128, 4: 64, 5: 128, 6: 85, 7: 85, 8: 85, 9: 128, 10: 85,
            11: 128, 12: 85}
    stream = torch.cuda.current_stream()
    n_steps = args.mpc_steps if args.mpc_steps > 6 else 9
    rows = []
    auto = None
    for v in (range(13) if args.variant < 0 else [args.variant]):
        sol = pkg.Solver(p)
        if auto is None:
            auto = pkg.tma_get_tuning(sol.h)[0]
        try:
            pkg.tma_set_tuning(sol.h, v)
        except pkg.TmaError:
            sol.close()
            continue
        sol.solve()                    # warm
        sol.set_state(mpc_step=0)
        ms = []
        for step in range(n_steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            pkg.tma_mpc_run(sol.h, 1, p.N)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        sol.close()
        rows.append({"variant": v, "layout": names[v], "threads_per_block": 32 * p.N,
                     "max_registers": regs[v], "ms_per_update_by_step": [round(x, 2) for x in ms],
                     "settled_ms_per_update": round(float(np.mean(ms[5:])), 3)})
    for r in rows:
        r["aircraft_step_samples_per_s"] = round(units_settled / (r["settled_ms_per_update"] * 1e-3), 1)
    best = min(rows, key=lambda r: r["settled_ms_per_update"]) if rows else None
    print(json.dumps({"mode": "layout-sweep",
                      "workload": "tma-10ac-enter5-L10240-H6-J100-schedule-corner-wind-rolling",
                      "draws_per_particle": draws, "units_per_settled_update": units_settled,
                      "autotuner_choice": auto, "rows": rows,
                      "paper": {"best_s": 56.0, "best_layout": "320x32", "used_s": 58.0,
                                "used_layout": "128x80", "hardware": "GeForce GTX 580"},
                      "speedup_vs_paper_best": (round(56.0 / (best["settled_ms_per_update"] * 1e-3), 1)
                                                if best else None)}), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="c3",
                    help="the timed workload: c3 the 24-aircraft high-density TMA (default), "
                         "c2 the 8-aircraft one")
    ap.add_argument("--e2e-steps", type=int, default=3,
                    help="solves of the end-to-end (host buffers) measurement, at most --steps")
    ap.add_argument("--cpu-particles", type=int, default=0,
                    help="particles of the oracle's CPU-baseline sample (0: the workload's)")
    ap.add_argument("--reference-particles", type=int, default=0,
                    help="particles per step of the reference arm (0: the workload's)")
    ap.add_argument("--rollout-only", action="store_true",
                    help="time only the rollout on --particles particles (profiling case)")
    ap.add_argument("--particles", type=int, default=0,
                    help="particles of the profiling / batched cases (0: the workload's own)")
    ap.add_argument("--batched", action="store_true",
                    help="time the batched MPC workload (graph-captured receding-horizon steps)")
    ap.add_argument("--scenarios", type=int, default=256)
    ap.add_argument("--single-sample", type=int, default=32,
                    help="--batched: scenarios of the one-solver-per-scenario comparison")
    ap.add_argument("--mpc-steps", type=int, default=10)
    ap.add_argument("--config", type=int, default=2,
                    help="workload of --rollout-only (1-4)")
    ap.add_argument("--samples", type=int, default=0,
                    help="--rollout-only: wind samples (0: the workload's own; fewer keep a profiling "
                         "case small)")
    ap.add_argument("--stages", action="store_true",
                    help="time normalisation, resampling and move alone on the 24-aircraft sizes")
    ap.add_argument("--stage", choices=("all", "lse", "resample", "lse_resample", "move"), default="all",
                    help="with --stages: time one stage only (the move's solver is allocated only for the move)")
    ap.add_argument("--late", action="store_true",
                    help="profiling cases: use the particles of a finished solve (late iterations)")
    ap.add_argument("--grad-only", action="store_true",
                    help="time only the gradient pass on --particles particles (profiling case)")
    ap.add_argument("--moves", action="store_true",
                    help="compare the paper's move with accepted random-walk and Langevin moves")
    ap.add_argument("--wind", choices=("shared", "corners", "own"), default="shared",
                    help="--rollout-only: the workload's shared field, a shared field on the 2x2x2 "
                         "corner grid, or every particle's own field on that grid")
    ap.add_argument("--schedule", action="store_true",
                    help="compare fixed work with the sample schedule (the inner loop of Algorithm 1) "
                         "and a falling particle count")
    ap.add_argument("--layout-sweep", action="store_true",
                    help="re-run the paper's thread/block layout sweep (forced launch variants)")
    ap.add_argument("--variant", type=int, default=-1,
                    help="with --layout-sweep: only this launch variant")
    ap.add_argument("--seeds", type=int, default=10)
    ap.add_argument("--eps-rw", type=float, default=1.0)
    ap.add_argument("--eps-mala", type=float, default=0.3)
    args = ap.parse_args(argv)
    world, rank, local = dist_setup()
    if args.rollout_only:
        return run_rollout_only(args, local)
    if args.batched:
        return run_batched(args, local)
    if args.moves:
        return run_moves(args, local)
    if args.schedule:
        return run_schedule(args, local)
    if args.layout_sweep:
        return run_layout_sweep(args, local)
    if args.grad_only:
        return run_grad_only(args, local)
    if args.stages:
        return run_stages(args, local)
    if args.impl == "reference":
        return run_reference(args, world, rank)
    return run_ours(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
