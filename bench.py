#!/usr/bin/env python
"""Benchmark: phase-shift RK2 steps/s and Gcells/s vs RK4 + 2/3 truncation at the same kmax.

Workload (timed `--steps` steps, one JSON line on rank 0):
  Taylor-Green vortex (Sec. 3.4, Eq. T-G-init), Re = 1/nu = 1600, 256^3, L = 2 pi,
  RK2 phase-shift random (Rogallo) with spherical truncation C_t = 1 (kmax = 128),
  FP32 butterflies and products, FP64 tables and reductions, dt from CFL 0.5 with the
  CFL frequency summed over directions (dt = 0.5 dx / 2 for this field) and rounded so
  that t = 9 lands on a step, shifts from splitmix64 seed 12345.
  Comparison leg: RK4 + 2/3 spherical truncation at 384^3 (kmax = 128, same dt rule).

Per step the state (201 MB) and the moved data (2.95 GB by the two-pass byte model) are
larger than the 129 MB L2, so no L2 flush is needed between steps.

--impl reference times the FP64 CPU oracle on the host cores on the same workload (a
bounded number of whole steps).  Under torchrun (N > 1) every rank runs an independent
replica (weak scaling, no collective on the data path) and value = all ranks' steps / the
slowest rank's time.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "phase-shift RK2 steps/s & Gcells/s vs RK4+2/3 at same kmax; % HBM roofline"
N_PS, N_RK4, KMAX, NU, SEED, CFL, T_END = 256, 384, 128.0, 1.0 / 1600.0, 12345, 0.5, 9.0
WORKLOAD = ("Taylor-Green Re=1600, 256^3, RK2 phase-shift random (Rogallo), spherical C_t=1 "
            "(kmax=128), FP32 bulk / FP64 reductions, dt = 0.5 / sum_i(max|u_i|/dx) (t=9 on a step)")


def dt_for(N):
    """dt = CFL / sum_i(max|u_i| / dx), rounded down so that t = 9 lands on a step.

    For the Taylor-Green field max|u_x| = max|u_y| = 1 and u_z = 0, so dt = CFL dx / 2.
    """
    dt = CFL / (2.0 / (2 * math.pi / N))
    return T_END / math.ceil(T_END / dt)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--rk4-steps", type=int, default=30)
    ap.add_argument("--e2e-steps", type=int, default=None,
                    help="steps of the end-to-end leg (default: --steps)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the cpu_baseline leg")
    ap.add_argument("--no-rk4", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the accuracy leg (PS 256^3 FP32/FP64 and RK4 384^3 to t = 9)")
    ap.add_argument("--batch-steps", type=int, default=200,
                    help="steps of the 64-member ensemble leg (0: skip)")
    ap.add_argument("--quality", action="store_true",
                    help="run the accuracy study at kmax = 108 instead (spectral error vs speedup)")
    ap.add_argument("--quality-cfl", action="store_true",
                    help="with --quality: adaptive CFL steps (0.4 for the RK2 family, 1.0 for RK4)")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("ns_fft.cuh", "ns_kernels.cuh", "ns_fft2.cuh", "ns_kernels2.cuh"):
        with open(os.path.join(ROOT, "paper_2603_08892_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel):
    """DRAM bytes per launch from the committed ncu summary, if it matches the kernels."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            d = json.load(f)
        if d.get("kernel_source_hash") != kernel_source_hash():
            return None
        return d["kernels"][kernel]["dram_bytes_per_launch_full_size"]
    except Exception:
        return None


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, local_rank):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        ids = [v for v in vis.split(",") if v.strip()]
        self.idx = ids[local_rank] if local_rank < len(ids) else str(local_rank)
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", self.idx, "--query-gpu=" + self.Q, "--format=csv,noheader",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.p is None:
            return out
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1].split()[0]))
                smax.append(float(parts[2].split()[0]))
            except Exception:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.f.name)
        if sm:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                   "reasons": sorted(reasons), "samples": len(sm)}
        return out


def reduce_max(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def host_cores():
    """(threads this process may use, CPU model name from lscpu)."""
    cores = len(os.sched_getaffinity(0))
    model = "unknown"
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return cores, model


def cpu_oracle_rate(budget_s=60.0, max_steps=3, warmup=0, seed=SEED):
    """Oracle steps/s on the workload (whole 256^3 steps, bounded by a wall-time budget), its
    3D transforms on every host core (scipy.fft workers).  Returns (rate, steps, seconds,
    final state)."""
    from oracle import rng as orng
    from oracle import schemes as sc
    from oracle import spectral as osp
    from paper_2603_08892_gb300 import inputs

    cores, _ = host_cores()
    old = osp.set_fft_workers(cores)
    try:
        N = N_PS
        dt = dt_for(N)
        prob = sc.Problem(N, NU, KMAX)
        S = osp.set_velocity(inputs.taylor_green(N), KMAX)
        for n in range(warmup):
            S = sc.step_ps_random(S, dt, prob, orng.shift_alpha(seed, n, N))
        t0 = time.perf_counter()
        n = 0
        while n < max_steps:
            S = sc.step_ps_random(S, dt, prob, orng.shift_alpha(seed, warmup + n, N))
            n += 1
            if time.perf_counter() - t0 > budget_s:
                break
        el = time.perf_counter() - t0
    finally:
        osp.set_fft_workers(old)
    return n / el, n, el, S


def run_reference(args, rank, world):
    if rank != 0:
        return
    steps = max(1, args.steps)
    rate, n, el, _ = cpu_oracle_rate(budget_s=150.0, max_steps=steps, warmup=min(args.warmup, 1))
    cores, model = host_cores()  # the 3D transforms use every core; elementwise work one
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": "steps/s",
        "n_gpus": args.gpus, "steps": n, "warmup": min(args.warmup, 1),
        "ms_per_step": 1000.0 * el / n, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (Taylor-Green field, Eq. T-G-init)",
        "config": {"workload": WORKLOAD + " -- FP64 CPU oracle", "N": N_PS, "dt": dt_for(N_PS)},
        "gcells_per_s": rate * N_PS ** 3 / 1e9,
        "cpu_baseline": {"value": rate, "unit": "steps/s", "cores": cores, "kind": "oracle",
                         "cpu_model": model,
                         "sample": "%d whole 256^3 steps after %d warm-up step(s), %.1f s (FP64 "
                                   "NumPy oracle, 3D transforms by scipy.fft on %d threads)"
                                   % (n, min(args.warmup, 1), el, cores)},
        "e2e": {"value": rate, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_quality(local, adaptive=False):
    """Accuracy / speed study at kmax = 108 (Sec. 5, Fig. quality, supplementary Table
    tab:quality): Taylor-Green Re = 1600 to t = 12 with the spectral error index (Eq. quality)
    of the 1D spectra over the window t = 7 .. 12 around the dissipation peak (t_end = t_start
    + 5), sampled at integer times, against RK4 at N = 324, C_t = 2/3.  FP32, time step
    1 / ceil(1 / (0.25 dx)) (CFL 0.5 reading, integer times on steps).  Speedup = GPU time of
    the reference run / GPU time of the run (stepping only, CUDA events).

    adaptive: every step from the CFL condition of the velocity its first evaluation forms
    (ns_step_cfl; the paper's coefficients, 0.4 for the RK2 family and 1.0 for RK4, Sec. 2),
    each step capped so that the run lands on the integer sampling times; the GPU time is the
    sum of the steps' event times (the host turnaround between the one-step calls excluded)."""
    import torch

    from paper_2603_08892_gb300 import analysis
    from paper_2603_08892_gb300 import binding as ns
    from paper_2603_08892_gb300 import inputs

    torch.cuda.set_device(local)
    kmax, T, t0 = 108.0, 12, 7
    cases = [("RK4 C_t=2/3 (reference)", 324, ns.RK4, ns.TRUNC_SPHERICAL),
             ("RK2 PS exact C_t=1 spherical", 216, ns.RK2_PS_EXACT, ns.TRUNC_SPHERICAL),
             ("RK2 PS random C_t=1 spherical", 216, ns.RK2_PS_RANDOM, ns.TRUNC_SPHERICAL),
             ("RK2 PS exact C_t=1 no double aliases", 216, ns.RK2_PS_EXACT, ns.TRUNC_NO_DOUBLE_ALIAS),
             ("RK2 PS random C_t=1 no double aliases", 216, ns.RK2_PS_RANDOM, ns.TRUNC_NO_DOUBLE_ALIAS),
             ("RK4 C_t=1 spherical (aliased)", 216, ns.RK4, ns.TRUNC_SPHERICAL),
             ("RK2 C_t=2/3 (time-step error only)", 324, ns.RK2, ns.TRUNC_SPHERICAL)]
    out, ref_spec, ref_ms = [], None, None
    for name, N, scheme, trunc in cases:
        dt = 1.0 / math.ceil(1.0 / (0.25 * 2 * math.pi / N))
        per = int(round(1.0 / dt))
        cfl = 1.0 if scheme == ns.RK4 else 0.4
        stream = torch.cuda.Stream()
        with ns.Solver(N, 1.0 / 1600, kmax, scheme=scheme, truncation=trunc, precision=ns.FP32,
                       stream=stream.cuda_stream, seed=12345) as s:
            s.set_velocity(inputs.taylor_green(N))
            spec, ms, nst = [], 0.0, 0
            for j in range(1, T + 1):
                if adaptive:
                    t, _ = s.time()
                    while t < j - 1e-12:
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        s.step_cfl(cfl, j - t, 1)
                        e1.record(stream)
                        e1.synchronize()
                        ms += e0.elapsed_time(e1)
                        nst += 1
                        t, _ = s.time()
                else:
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    torch.cuda.synchronize()
                    e0.record(stream)
                    s.step(dt, per)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ms += e0.elapsed_time(e1)
                    nst += per
                if j >= t0:
                    spec.append(tuple(s.spectrum(k, 112) for k in (1, 2, 3)))
            E, eps = s.energy()
        if ref_spec is None:
            ref_spec, ref_ms = spec, ms
        out.append({"run": name, "N": N, "steps": nst, "dt": (T / nst) if adaptive else dt,
                    "cfl": cfl if adaptive else None, "gpu_s": ms / 1000.0,
                    "speedup": ref_ms / ms, "error_pct": analysis.error_index(spec, ref_spec, kmax),
                    "E_end": E, "eps_end": eps})
        print(json.dumps(out[-1]), flush=True)
    print(json.dumps({"study": "quality", "adaptive_cfl": adaptive, "kmax": kmax, "Re": 1600,
                      "window": [t0, T], "runs": out}))


def accuracy_leg(ns, inputs, stream, local, line):
    """Runs to t = 9: PS random 256^3 FP32 and FP64, RK4 + 2/3 384^3 FP32 (same kmax = 128).
    Returns E(9), eps(9) of each run, the error index of the PS run against RK4 and of FP32
    against FP64, and the simulated time per second of both schemes with the index beside it."""
    import torch

    from paper_2603_08892_gb300 import analysis

    runs = {}
    for name, N, scheme, prec in (("ps_fp32", N_PS, ns.RK2_PS_RANDOM, ns.FP32),
                                  ("ps_fp64", N_PS, ns.RK2_PS_RANDOM, ns.FP64),
                                  ("rk4_fp32", N_RK4, ns.RK4, ns.FP32)):
        dtn = dt_for(N)
        nsteps = int(round(T_END / dtn))
        with ns.Solver(N, NU, KMAX, scheme=scheme, precision=prec, device=local,
                       stream=stream.cuda_stream, seed=SEED) as r:
            r.set_velocity(inputs.taylor_green(N))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            r.step(dtn, nsteps)
            e1.record(stream)
            torch.cuda.synchronize()
            t, _ = r.time()
            E, eps = r.energy()
            spec = tuple(r.spectrum(k, 130) for k in (1, 2, 3))
        runs[name] = {"N": N, "steps": nsteps, "t": t, "E": E, "eps": eps,
                      "gpu_s": e0.elapsed_time(e1) / 1000.0, "spec": spec}
    ps, ps64, rk = runs["ps_fp32"], runs["ps_fp64"], runs["rk4_fp32"]
    err_rk4 = analysis.error_index([ps["spec"]], [rk["spec"]], KMAX)
    err_64 = analysis.error_index([ps["spec"]], [ps64["spec"]], KMAX)
    sim_ps = line["sim_time_per_s"]
    sim_rk = line.get("rk4_two_thirds", {}).get("sim_time_per_s", T_END / rk["gpu_s"])
    out = {"t_end": T_END,
           "error_index_vs_rk4_pct": err_rk4,
           "error_index_fp32_vs_fp64_pct": err_64,
           "E9": {k: v["E"] for k, v in runs.items()},
           "eps9": {k: v["eps"] for k, v in runs.items()},
           "E9_fp32_vs_fp64_rel": abs(ps["E"] - ps64["E"]) / ps64["E"],
           "steps_to_t9": {k: v["steps"] for k, v in runs.items()},
           "gpu_s_to_t9": {k: v["gpu_s"] for k, v in runs.items()},
           "sim_time_per_s": {"ps_fp32_256": sim_ps, "rk4_fp32_384": sim_rk},
           "sim_time_speedup_vs_rk4": sim_ps / sim_rk,
           "what": "PS random 256^3 FP32 delivers sim_time_speedup_vs_rk4 times the simulated "
                   "time per second of RK4 + 2/3 at 384^3 (same kmax), at a spectral error "
                   "index error_index_vs_rk4_pct (%) against it at t = 9"}
    return out


def timed_steps(ns, s, dt, K, stream):
    import torch

    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    s.step(dt, K)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.quality:
        if rank == 0:
            run_quality(local, adaptive=args.quality_cfl)
        return
    import numpy as np
    import torch

    from paper_2603_08892_gb300 import binding as ns
    from paper_2603_08892_gb300 import inputs

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.Stream()
    W = max(3, args.warmup)
    K = max(1, args.steps)
    dt = dt_for(N_PS)
    # the input field in pinned host memory (a page-locked torch buffer viewed as NumPy)
    u0_pin = torch.empty((3, N_PS, N_PS, N_PS), dtype=torch.float64, pin_memory=True)
    u0 = u0_pin.numpy()
    u0[...] = inputs.taylor_green(N_PS)

    s = ns.Solver(N_PS, NU, KMAX, scheme=ns.RK2_PS_RANDOM, precision=ns.FP32, device=local,
                  stream=stream.cuda_stream, seed=SEED + rank)
    s.set_velocity(u0)
    s.step(dt, W)
    clocks = Clocks(local)
    barrier(world)
    clocks.start()
    ms = timed_steps(ns, s, dt, K, stream)  # the headline: no per-kernel instrumentation
    clk = clocks.stop()
    E, eps = s.energy()
    # per-kernel CUDA-event times from a separate instrumented run (one chunk of Kp steps)
    Kp = min(K, 200)
    s.profile(True)
    timed_steps(ns, s, dt, Kp, stream)
    prof = s.profile_read()
    s.profile(False)
    # adaptive CFL stepping (paper's coefficient 0.4 for RK2 schemes): one read-back per step
    Ka = 200
    t_a0, _ = s.time()
    ea0 = torch.cuda.Event(enable_timing=True)
    ea1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ea0.record(stream)
    s.step_cfl(0.4, 1.0, Ka)
    ea1.record(stream)
    torch.cuda.synchronize()
    t_a1, _ = s.time()
    adaptive = {"cfl": 0.4, "steps": Ka, "steps_per_s": Ka / (ea0.elapsed_time(ea1) / 1000.0),
                "mean_dt": (t_a1 - t_a0) / Ka, "fixed_dt": dt}
    # diagnostic cost: flux and cumulative dissipation with the two-shift average (ns_energy_flux)
    dxq = 2 * math.pi / N_PS
    s.energy_flux(200, [[0, 0, 0], [dxq / 2] * 3])
    torch.cuda.synchronize()
    tf0 = time.perf_counter()
    s.energy_flux(200, [[0, 0, 0], [dxq / 2] * 3])
    flux_ms = (time.perf_counter() - tf0) * 1000.0
    ms_max = reduce_max(ms, world)
    barrier(world)

    C = N_PS ** 3 * 4.0
    model_bytes = s.model_bytes_per_step()
    value = world * K / (ms_max / 1000.0)
    ms_step = ms_max / K
    hbm, peak_kind = peaks()

    # Roofline units.  The pencil pass is one launch (2 per step).  The slab pass is three
    # kernels per plane group (y inverse, x rows, y forward) whose algorithmic traffic is the
    # 5 mixed fields read (5C) and the 3 transformed products written (3C), 8C per pass; its
    # scratch is an implementation choice (L2 or HBM by group size) and shows in the measured
    # ncu traffic, not in the model.
    nchunks = (K + 255) // 256
    # every pencil pass of a step reads Ft and the state and writes the state and the mixed
    # fields of the next evaluation (the last one prepares the next step): 14C per launch
    units = {
        "k_pencil": (14.0 * C, prof["k_pencil"][0], prof["k_pencil"][1]),
        "slab_pass": (8.0 * C, prof["slab_pass"][0], prof["slab_pass"][1]),
    }
    roof_units = {}
    for name, (nbytes, tot_ms, n) in units.items():
        avg = tot_ms / max(1, n)
        ach = nbytes / (avg / 1000.0) / 1e9
        roof_units[name] = {"algorithmic_bytes_per_launch": nbytes, "avg_launch_ms": avg,
                            "achieved": ach, "frac": ach / hbm, "ms_per_step": tot_ms / Kp}
    dom = max(roof_units, key=lambda k: roof_units[k]["ms_per_step"])
    kern = ("k_pencil", "k_yinv", "k_xrow", "k_yfwd")
    tot = {k: prof[k][0] for k in kern}
    # time breakdown of the step by pass (events on the stepping stream; the two sum to about
    # the step time); the per-kernel event times overlap (the slab groups run on two streams,
    # so each kernel's events also span the other stream's concurrent work) and do not add up
    pass_ms = {k: round(roof_units[k]["ms_per_step"], 4) for k in roof_units}
    pass_shares = {k: round(v / max(1e-9, sum(pass_ms.values())), 4) for k, v in pass_ms.items()}
    kernel_ms = {k: round(tot[k] / Kp, 4) for k in tot}
    # launches in the timed region: the kernels per step from the instrumented run (the mixed
    # fields carried from the previous call spare the INIT pass), plus the shift-table kernel
    # of every chunk of 256 steps
    per_step = sum(prof[k][2] for k in kern) / Kp
    launches = int(round(per_step * K)) + nchunks
    ru = roof_units[dom]
    roof = {"bound": "hbm",
            "kernel": dom if dom == "k_pencil" else "slab_pass (k_yinv + k_xrow + k_yfwd)",
            "achieved": ru["achieved"], "peak": hbm, "unit": "GB/s", "frac": ru["frac"],
            "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)",
            "algorithmic_bytes_per_launch": ru["algorithmic_bytes_per_launch"],
            "avg_launch_ms": ru["avg_launch_ms"], "traffic": ncu_traffic(dom),
            "units": roof_units, "pass_ms_per_step": pass_ms, "pass_time_shares": pass_shares,
            "kernel_event_ms_per_step_overlapping": kernel_ms,
            "slab_groups_per_pass": prof["k_yinv"][2] / max(1, prof["slab_pass"][2]),
            "step_model_bytes": model_bytes,
            "step_frac": (model_bytes / (ms_step / 1000.0) / 1e9) / hbm}

    # secondary roofline: FP32 CUDA-core arithmetic, 130 N^3 log2 N flop per RK2-family step
    # (radix-2 operation count of the step's 3D transforms) against the measured FMA peak
    fma32 = ns.fma_peak(ns.FP32, device=local)
    fma64 = ns.fma_peak(ns.FP64, device=local)
    step_flops = 130.0 * N_PS ** 3 * math.log2(N_PS)
    alu = {"bound": "alu", "flops_per_step": step_flops,
           "achieved": step_flops / (ms_step / 1000.0) / 1e12, "peak": fma32 / 1e12,
           "unit": "TFLOP/s", "frac": step_flops / (ms_step / 1000.0) / fma32,
           "peak_source": "measured (ns_fma_peak, FP32 FMA chains on every SM)",
           "fp64_fma_peak_tflops": fma64 / 1e12}

    line = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (Taylor-Green initial field, Eq. T-G-init; no dataset)",
        "config": {"workload": WORKLOAD, "N": N_PS, "kmax": KMAX, "nu": NU, "dt": dt,
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "no flush: state 201 MB and 2.95 GB moved per step exceed the 129 MB L2"},
        "gcells_per_s": value * N_PS ** 3 / 1e9,
        "sim_time_per_s": value * dt / world,
        "energy_at_end": E, "dissipation_at_end": eps,
        "roofline": roof, "alu_roofline": alu, "gpu_launches": launches, "clocks": clk,
        "diagnostics_ms": {"energy_flux_two_shifts": flux_ms}, "adaptive_cfl": adaptive,
    }

    # RK4 + 2/3 truncation at 384^3, same kmax (comparison leg)
    if not args.no_rk4:
        dt4 = dt_for(N_RK4)
        r = ns.Solver(N_RK4, NU, KMAX, scheme=ns.RK4, precision=ns.FP32, device=local,
                      stream=stream.cuda_stream)
        r.set_velocity(inputs.taylor_green(N_RK4))
        r.step(dt4, 2)
        Kr = max(3, args.rk4_steps)
        ms4 = reduce_max(timed_steps(ns, r, dt4, Kr, stream), world)
        rate4 = world * Kr / (ms4 / 1000.0)
        mb4 = r.model_bytes_per_step()
        line["rk4_two_thirds"] = {
            "N": N_RK4, "kmax": KMAX, "dt": dt4, "steps": Kr, "steps_per_s": rate4,
            "gcells_per_s": rate4 * N_RK4 ** 3 / 1e9, "sim_time_per_s": rate4 * dt4 / world,
            "ms_per_step": ms4 / Kr, "step_frac_hbm": (mb4 / (ms4 / Kr / 1000.0) / 1e9) / hbm}
        line["sim_time_speedup_vs_rk4"] = line["sim_time_per_s"] / line["rk4_two_thirds"]["sim_time_per_s"]
        r.close()

    # accuracy beside the speed (config 2): the 256^3 Rogallo run in FP32 and FP64 and the 384^3
    # RK4 + 2/3 run to t = 9 (the Taylor-Green dissipation peak), the spectral error index of
    # Sec. 3.4 (Eq. quality, Appendix A) of the 1D spectra at t = 9
    if rank == 0 and world == 1 and not args.no_accuracy:
        line["accuracy_t9"] = accuracy_leg(ns, inputs, stream, local, line)

    # batched ensemble: 64 Taylor-Green members with 1% perturbations, 16 each of
    # N = 32, 64, 96, 128, Rogallo RK2 FP32, schedule chosen by the batch's tuner (one
    # persistent launch per call, or one grid launch per pass and size class)
    if args.batch_steps > 0:
        Ns = [32] * 16 + [64] * 16 + [96] * 16 + [128] * 16
        dts = [0.5 * (2 * math.pi / n) / 2.0 for n in Ns]
        b = ns.Batch(Ns, [NU] * len(Ns), [n / 2.0 for n in Ns], seeds=list(range(len(Ns))),
                     scheme=ns.RK2_PS_RANDOM, precision=ns.FP32, stream=stream.cuda_stream)
        for i, n in enumerate(Ns):
            b.set_velocity(i, inputs.taylor_green_perturbed(n, i))
        b.step(dts, 3)
        Kb = args.batch_steps
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.step(dts, Kb)
        e1.record(stream)
        torch.cuda.synchronize()
        msb = reduce_max(e0.elapsed_time(e1), world)
        Eb, _ = b.energy()
        gran, qsm = b.schedule()
        model = sum(44.0 * n ** 3 * 4.0 for n in Ns)
        line["batched_ensemble"] = {
            "members": len(Ns), "sizes": "16 x {32, 64, 96, 128}", "steps": Kb,
            "member_steps_per_s": world * len(Ns) * Kb / (msb / 1000.0),
            "ensemble_steps_per_s": world * Kb / (msb / 1000.0), "ms_per_step": msb / Kb,
            "schedule": {"kind": "grid" if gran == 0 else "persistent", "tiles_per_ticket": gran,
                         "ctas_per_sm": qsm},
            "launches_per_call": 4 * (2 + 9 * Kb) if gran == 0 else 1,
            "persistent_ctas": b.grid() if gran != 0 else None,
            "gcells_per_s": world * sum(n ** 3 for n in Ns) * Kb / (msb / 1000.0) / 1e9,
            "model_bytes_per_step": model,
            "frac_hbm": (model / (msb / Kb / 1000.0) / 1e9) / hbm,
            "frac_alu": sum(130.0 * n ** 3 * math.log2(n) for n in Ns) / (msb / Kb / 1000.0) / fma32,
            "finite": bool(np.all(np.isfinite(Eb)))}
        b.close()

    # end to end through the C ABI with host buffers: the host velocity in once, then E and eps
    # of every step to the host (ns_step_diag: one 16-byte copy per step, no host
    # synchronisation per step)
    Ke = max(3, K if args.e2e_steps is None else min(args.e2e_steps, K))
    s.set_velocity(u0)  # warm-up calls (the first call after the other legs pays one-time costs)
    s.step(dt, 1)
    s.step_diag(dt, 1)  # allocates the series buffers outside the timed region
    barrier(world)
    torch.cuda.synchronize()
    u_out = torch.empty((3, N_PS, N_PS, N_PS), dtype=torch.float64, pin_memory=True).numpy()
    s.get_velocity(u_out)  # (warm-up of the read-back path)
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.set_velocity(u0)  # synchronises
    t1 = time.perf_counter()
    Es, epss = s.step_diag(dt, Ke)
    t2 = time.perf_counter()
    s.get_velocity(u_out)  # the final velocity back to pinned host memory (synchronises)
    t3 = time.perf_counter()
    el = reduce_max(t3 - t0, world)
    h2d = (3 * N_PS ** 3 * 8 + Ke * 48) / Ke  # the FP64 field once, the shift vectors per step
    d2h = (Ke * 16 + 3 * N_PS ** 3 * 8) / Ke  # E and eps per step, the FP64 field once
    line["e2e"] = {"value": world * Ke / el, "unit": "steps/s", "h2d_bytes_per_step": h2d,
                   "d2h_bytes_per_step": d2h, "set_velocity_ms": (t1 - t0) * 1000.0,
                   "step_diag_ms_per_step": (t2 - t1) * 1000.0 / Ke,
                   "get_velocity_ms": (t3 - t2) * 1000.0,
                   "finite": bool(np.all(np.isfinite(Es)) and np.all(np.isfinite(epss))
                                  and np.all(np.isfinite(u_out))),
                   "what": "ns_set_velocity(pinned host 3x256^3 f64) + ns_step_diag(dt, %d): E and eps "
                           "of every step written by the device into mapped pinned host memory as "
                           "it is produced + ns_get_velocity(final field to pinned host f64); %d steps"
                           % (Ke, Ke)}
    # the same with a host round trip every step: ns_step(dt, 1) then ns_energy
    Ks = min(Ke, 200)
    s.set_velocity(u0)
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    for _ in range(Ks):
        s.step(dt, 1)
        s.energy()
    t4 = time.perf_counter()
    line["e2e"]["sync_every_step"] = {"steps": Ks, "step_and_energy_ms": (t4 - t3) * 1000.0 / Ks,
                                      "steps_per_s": Ks / reduce_max(t4 - t3, world)}
    s.close()

    if rank == 0 and world == 1 and not args.no_cpu:
        rate, n, el, S_ref = cpu_oracle_rate(budget_s=40.0, max_steps=3)
        cores, model = host_cores()
        line["cpu_baseline"] = {"value": rate, "unit": "steps/s", "cores": cores, "kind": "oracle",
                                "cpu_model": model,
                                "sample": "%d whole 256^3 Rogallo steps of the FP64 NumPy oracle "
                                          "(3D transforms by scipy.fft on %d threads), %.1f s"
                                          % (n, cores, el)}
        # the sampled oracle steps double as a parity check of the benchmarked kernels: the
        # same steps on the GPU (FP32 and FP64) from the same field, whole-state relative L2
        errs = {}
        for prec, name in ((ns.FP32, "fp32"), (ns.FP64, "fp64")):
            with ns.Solver(N_PS, NU, KMAX, scheme=ns.RK2_PS_RANDOM, precision=prec, device=local,
                           seed=SEED) as g:
                g.set_velocity(inputs.taylor_green(N_PS))
                g.step(dt, n)
                got = g.get_state()
            errs["rogallo_%d_steps_256_%s" % (n, name)] = float(
                np.linalg.norm(got - S_ref) / np.linalg.norm(S_ref))
        line["precision_errors"] = {
            "vs": "FP64 oracle, the cpu_baseline sample's steps, whole state, relative L2",
            "bounds": {"fp32_per_step": 2e-5, "fp64_per_step": 1e-12}, **errs}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
