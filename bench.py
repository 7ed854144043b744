#!/usr/bin/env python
"""Benchmark of the exact spherical-polar Poisson solve (Mueller & Chan 2018) on GB300.

One step = one whole solve Phi = L^-1 (4 pi G rho) of the 550x128x256 stellar workload
(log-stretched r, seeded l<=20 spherical-harmonic perturbation), inputs resident in HBM.
Prints one JSON line (rank 0).  `value` is zones/s of the headline precision; the
float64 path is reported beside it.  With --impl reference the CPU oracle is timed on
the host cores instead (a deliberately slow baseline).

Launch: python bench.py [--gpus N --steps K --warmup W]; for N>1 under torchrun each
rank solves its own instance (independent problems, no collective on the data path)."""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "zones/s at 550x128x256, mixed vs FP64 @1e-10 rel err; served p50/p99 latency"
WORKLOAD = "stellar_sh 550x128x256 (log r in [1e-3,1] with origin cell, uniform theta/phi, l<=20 SH perturbation, seed 3)"
PAPER_BEST_ZPS = 18022400 / 0.036   # Table 1: parity-split solver, 1024 Magnus CPU cores


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "mixed", "mixed_x3"], default=None,
                    help="headline arithmetic: mixed = 6-product split bf16 (default), mixed_x3 = 3-product")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-oracle-check", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 64-instance ragged batch")
    ap.add_argument("--no-served", action="store_true", help="skip the served Poisson-arrival stream")
    ap.add_argument("--served-requests", type=int, default=400)
    ap.add_argument("--no-small", action="store_true", help="skip the 32x16x32 and 128x64x128 configurations")
    ap.add_argument("--autotune", action="store_true",
                    help="tune each plan's launch configuration (sp_plan_autotune) before timing")
    ap.add_argument("--headline-only", action="store_true",
                    help="time the headline precision only (no float64 / 3-product comparison plans)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------ multi-rank
def max_over_ranks(x, world, device):
    """Largest value of x over all ranks of the default process group (x itself for one
    rank): the job's time is its slowest rank's."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank_step, steps, world, seconds):
    """Units processed by all ranks per second of the slowest rank (weak scaling: every
    rank solves its own instance)."""
    return units_per_rank_step * steps * world / seconds


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int, period_ms: int = 20):
        self.dev = device_index
        self.period_ms = period_ms
        self.proc = None
        self.path = None

    def start(self):
        """Start sampling (nvidia-smi in the background, one line per period)."""
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu=timestamp,{self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", str(self.period_ms)],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)   # the first sample lands before the work starts

    def stop(self, window=None):
        """Median SM clock and active throttle reasons over the samples; `window` = (t0, t1)
        wall-clock seconds of the timed region, whose samples are counted separately."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons, in_win = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                mhz, mx = float(f[2]), float(f[3])
            except ValueError:
                continue
            sm.append(mhz)
            smax.append(mx)
            for nm, v in zip(names, f[6:10]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
            if window is not None:
                try:
                    import datetime
                    ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                    if window[0] <= ts <= window[1]:
                        in_win.append(mhz)
                except ValueError:
                    pass
        os.unlink(self.path)
        out = {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
               "reasons": sorted(reasons), "samples": len(sm), "period_ms": self.period_ms,
               "span": "warm-up, timed steps and the per-kernel pass of the headline plan"}
        if window is not None:
            out["samples_in_timed_steps"] = len(in_win)
            out["sm_mhz_in_timed_steps"] = statistics.median(in_win) if in_win else None
        return out


# ------------------------------------------------------------ CPU baseline
def oracle_zones_per_s(budget_s: float = 12.0):
    """The CPU oracle (float64 NumPy/SciPy, as it stands) on the bench workload, repeated
    until `budget_s` of CPU work; returns (zones/s, solves, seconds)."""
    import workloads as W
    from oracle import sph_poisson as O
    p = W.stellar_sh()
    geo = O.Geometry(p.r_if, p.th_if, p.nphi)
    n, t0 = 0, time.perf_counter()
    while True:
        O.solve_separated(geo, p.rho)
        n += 1
        el = time.perf_counter() - t0
        if el >= budget_s:
            break
    return p.zones * n / el, n, el


def cpu_cores():
    return os.cpu_count() or 1


def run_reference(args, rank):
    """Reference arm: the CPU oracle, one full solve of the workload per step."""
    if rank != 0:
        return
    import workloads as W
    from oracle import sph_poisson as O
    p = W.stellar_sh()
    geo = O.Geometry(p.r_if, p.th_if, p.nphi)
    for _ in range(args.warmup):
        O.solve_separated(geo, p.rho)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.solve_separated(geo, p.rho)
    el = time.perf_counter() - t0
    v = p.zones * args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "zones/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "global_batch": 1, "l2": "inputs larger than L2 (CPU run)"},
        "cpu_baseline": {"value": v, "unit": "zones/s", "cores": cpu_cores(), "kind": "oracle",
                         "sample": f"{args.steps} full float64 oracle solves of the workload"},
        "e2e": {"value": v, "unit": "zones/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
def run_ours(args, rank, world, local):
    import torch
    import paper_1806_06623_gb300 as S
    import workloads as W

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    S.lib()
    precision = args.precision or "mixed"
    p = W.stellar_sh()
    zones = p.zones
    rho = torch.from_numpy(p.rho).to(dev)
    phi = torch.empty_like(rho)
    stream = torch.cuda.current_stream(dev)

    plans = {}
    if precision == "fp64" or not args.headline_only:
        plans["fp64"] = S.Plan(p.r_if, p.th_if, p.nphi, precision=S.SP_FP64)
    if precision == "mixed_x3" or (precision == "mixed" and not args.headline_only):
        plans["mixed_x3"] = S.Plan(p.r_if, p.th_if, p.nphi, precision=S.SP_MIXED_BF16X3, tol=1e-10)
    if precision == "mixed":
        plans["mixed"] = S.Plan(p.r_if, p.th_if, p.nphi, precision=S.SP_MIXED_BF16X6, tol=1e-10)
    if precision == "mixed" and not args.headline_only:
        # the same 6-product solve refined with a float64 iterate and the float64 stencil
        plans["mixed_f64_residual"] = S.Plan(p.r_if, p.th_if, p.nphi, precision=S.SP_MIXED_BF16X6, tol=1e-10)
        plans["mixed_f64_residual"].set_residual(S.SP_RESIDUAL_FLOAT64)
    head = plans[precision]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    def timed_steps(plan, k, collect):
        tot = 0.0
        infos = []
        for _ in range(k):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, info = plan.solve(rho, phi)
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
            infos.append(info.as_dict())
            if collect:
                plan.collect_timing()
        return tot, infos

    tuning = {}
    if args.autotune:
        # launch configuration per plan from timed solves of this workload (sp_plan_autotune)
        for name, plan in plans.items():
            _, conf = plan.autotune(rho, phi)
            tuning[name] = dict(zip(("fft_lines_per_cta", "radix_order", "projection_ctas", "scan_components"), conf))
    results = {}
    for name, plan in plans.items():
        clocks = ClockSampler(local)
        if name == precision:
            clocks.start()
        for _ in range(args.warmup):
            plan.solve(rho, phi)
        barrier()
        n0 = plan.launch_count()
        barrier()
        w0 = time.time()
        tot_ms, infos = timed_steps(plan, args.steps, collect=False)
        barrier()
        w1 = time.time()
        launches = plan.launch_count() - n0
        # per-kernel breakdown in a separate pass: the per-launch CUDA events stay out of
        # the timed steps above
        nb = min(args.steps, 5)
        plan.set_timing(True)   # also clears the accumulators
        timed_steps(plan, nb, collect=True)
        timing = {k: (v[0] * args.steps / nb, v[1] * args.steps // nb) for k, v in plan.timing().items()}
        plan.set_timing(False)
        ck = clocks.stop(window=(w0, w1)) if name == precision else None
        tot_ms = max_over_ranks(tot_ms, world, dev)
        results[name] = {"ms": tot_ms, "infos": infos, "launches": launches, "timing": timing, "clocks": ck,
                         "phi": phi.detach().cpu().numpy() if (rank == 0 and not args.no_oracle_check) else None}

    # the acceleration on the faces (sp_face_gradients) of the solved potential: float64,
    # reads Phi (8 B per zone) and writes the r, theta and phi face gradients (8 B per face)
    face = None
    if rank == 0:
        fplan = plans.get("fp64", head)
        g = fplan.face_gradients(phi)
        torch.cuda.synchronize(dev)
        reps = 10
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            g = fplan.face_gradients(phi)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / reps
        nbytes = 8 * (phi.numel() + sum(x.numel() for x in g))
        try:
            pk = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6800.0))
        except Exception:
            pk = 6800.0
        face = {"ms": ms, "algorithmic_bytes": nbytes, "frac": nbytes / (ms / 1e3) / 1e9 / pk,
                "note": "float64 face gradients of Phi on the r, theta and phi faces (boundary faces through "
                        "the outer and inner conditions), L2 not flushed between the 10 calls"}
        del g

    # end-to-end through the host-buffer entry points (page-locked buffers, copies timed):
    # K solves in one pipelined call (the upload of step k+1 and the download of step k-1
    # overlap the solve of step k), and K single sp_solve_host calls (copy, solve, copy)
    rho_h = torch.from_numpy(p.rho).pin_memory()
    phi_h = torch.empty(p.rho.shape, dtype=torch.float64).pin_memory()
    rho_np, phi_np = rho_h.numpy(), phi_h.numpy()
    head.solve_host_pipelined([rho_np] * max(2, args.warmup), [phi_np] * max(2, args.warmup))
    barrier()
    t0 = time.perf_counter()
    head.solve_host_pipelined([rho_np] * args.steps, [phi_np] * args.steps)
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, world, dev)
    for _ in range(max(1, args.warmup // 2)):
        head.solve_host(rho_np, phi_np)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        head.solve_host(rho_np, phi_np)
    e2e_single_s = time.perf_counter() - t0
    e2e_single_s = max_over_ranks(e2e_single_s, world, dev)
    # the link's own rate for the same buffers: one step's H2D and D2H copies alone, one
    # after the other on one stream, and both directions at once on two streams
    d_tmp = torch.empty_like(rho)
    d_tmp2 = torch.empty_like(rho)
    phi_h2 = torch.empty_like(phi_h).pin_memory()
    torch.cuda.synchronize(dev)
    c0 = time.perf_counter()
    for _ in range(args.steps):
        d_tmp.copy_(rho_h, non_blocking=True)
        phi_h.copy_(d_tmp, non_blocking=True)
    torch.cuda.synchronize(dev)
    copy_s = (time.perf_counter() - c0) / args.steps
    s_up, s_down = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    torch.cuda.synchronize(dev)
    c0 = time.perf_counter()
    for _ in range(args.steps):
        with torch.cuda.stream(s_up):
            d_tmp.copy_(rho_h, non_blocking=True)
        with torch.cuda.stream(s_down):
            phi_h2.copy_(d_tmp2, non_blocking=True)
    torch.cuda.synchronize(dev)
    copy_both_s = (time.perf_counter() - c0) / args.steps
    # the same two copies beside an unrelated device solve (no dependencies between the
    # three): what the GPU gives a pipelined step, since copies and solve share it
    phi_d = torch.empty_like(rho)
    torch.cuda.synchronize(dev)
    c0 = time.perf_counter()
    for _ in range(args.steps):
        with torch.cuda.stream(s_up):
            d_tmp.copy_(rho_h, non_blocking=True)
        with torch.cuda.stream(s_down):
            phi_h2.copy_(d_tmp2, non_blocking=True)
        head.solve(rho, phi_d)
    torch.cuda.synchronize(dev)
    overlap_s = (time.perf_counter() - c0) / args.steps
    del d_tmp, d_tmp2, phi_d

    if rank != 0:
        return
    r = results[precision]
    value = whole_job_rate(zones, args.steps, world, r["ms"] / 1e3)
    line = {
        "metric": METRIC, "value": value, "unit": "zones/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": value / PAPER_BEST_ZPS,
        "vs_baseline_ref": "Table 1 of the paper: 0.036 s per 550x128x256 solve, parity-split, 1024 CPU cores",
        "dtype": {"fp64": "f64", "mixed_x3": "bf16 (2-plane split, 3 products) + f32, float-float refinement",
                  "mixed": "bf16 (3-plane split, 6 products) + f32, float-float refinement"}[precision],
        "tol": 1e-10,
        "solve_info": r["infos"][-1],
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": precision, "global_batch": world,
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": "flushed (256 MB write) between timed steps"},
        "clocks": r["clocks"],
        "gpu_launches": r["launches"],
        "e2e": {"value": whole_job_rate(zones, args.steps, world, e2e_s), "unit": "zones/s",
                "h2d_bytes_per_step": int(p.rho.nbytes), "d2h_bytes_per_step": int(p.rho.nbytes),
                "api": "sp_solve_host_pipelined: K solves from page-locked host buffers in one call",
                "ms_per_step": 1e3 * e2e_s / args.steps,
                "single_call_value": whole_job_rate(zones, args.steps, world, e2e_single_s),
                "single_call_api": "sp_solve_host per step (copy in, solve, copy out)",
                "copy_ms_per_step": 1e3 * copy_s,
                "copy_ms_per_step_both_directions_at_once": 1e3 * copy_both_s,
                "copy_bound_zones_per_s": zones / copy_both_s,
                "copies_beside_solve_ms_per_step": 1e3 * overlap_s,
                "note": "copy_ms_per_step: the step's H2D then D2H on one stream; both directions at once "
                        "(two streams) bound a pipelined step from below; copies_beside_solve: both "
                        "directions and an independent device solve at once (the device-to-host copy "
                        "slows under the solve's memory traffic), the bound a pipelined step meets"},
        "kernel_ms_per_step": {k: v[0] / args.steps for k, v in r["timing"].items()},
        "kernel_ms_note": "per-kernel-group CUDA-event spans of a separate timing pass (kernels launched one "
                          "by one); residual_rows is the residual's interior-row kernel, a span inside residual",
    }
    for name, rr in results.items():
        line[f"{name}_zones_per_s"] = whole_job_rate(zones, args.steps, world, rr["ms"] / 1e3)
        line[f"{name}_ms_per_step"] = rr["ms"] / args.steps
        line[f"{name}_iterations"] = rr["infos"][-1].get("iterations")
    line["roofline"] = roofline(r["timing"], p, precision, args.steps, r["infos"][-1].get("iterations", 2),
                                sm_mhz=(r["clocks"] or {}).get("sm_mhz"),
                                num_sms=torch.cuda.get_device_properties(dev).multi_processor_count)
    line["roofline_groups"] = roofline_groups(r["timing"], p, precision, args.steps,
                                              r["infos"][-1].get("iterations", 2))
    line["projection_tensor"] = projection_tensor_rate(r["timing"], p, precision)
    line["kernel_source_sha"] = kernel_source_hash()
    if face is not None:
        line["face_gradients"] = face
    line["autotuned"] = tuning or None
    # the served stream first: measured after the oracle's CPU checks in the same process
    # (small configurations, batch samples) it ran 15-40% slower, cause not isolated
    if not args.no_served:
        line["served"] = run_served(S, W, torch, args.served_requests)
    if not args.no_small:
        line["small_configs"] = run_small(S, W, torch, dev, check=not args.no_oracle_check)
    if not args.no_batched:
        line["batched"] = run_batched(S, W, torch, dev, check=not args.no_oracle_check)
    if not args.no_oracle_check:
        line["error_vs_oracle"] = check_vs_oracle(p, {k: v["phi"] for k, v in results.items()})
    if not args.no_cpu_baseline and args.gpus == 1:
        zps, n, el = oracle_zones_per_s()
        line["cpu_baseline"] = {"value": zps, "unit": "zones/s", "cores": cpu_cores(), "kind": "oracle",
                                "sample": f"{n} full float64 oracle solves of the workload in {el:.1f} s "
                                          "(NumPy FFT and Thomas single-threaded, BLAS matmul multi-threaded)"}
    print(json.dumps(line), flush=True)


def run_small(S, W, torch, dev, check=True, steps=20, warmup=3):
    """The two smaller configurations (32x16x32 sphere, 128x64x128 stellar noise): one
    solve per step, float64 and 6-product mixed; these fit in L2, so the numbers are
    L2-resident rates (no flush between steps)."""
    out = {}
    for make in (W.sphere_blob, W.stellar_noise):
        p = make()
        rho = torch.from_numpy(p.rho).to(dev)
        phi = torch.empty_like(rho)
        stream = torch.cuda.current_stream(dev)
        key = "x".join(str(v) for v in p.shape)
        res = {"zones": p.zones, "l2": "resident (inputs smaller than L2)"}
        ref = None
        if check:
            from oracle import sph_poisson as O
            ref = O.solve_separated(O.Geometry(p.r_if, p.th_if, p.nphi), p.rho)
        for name, prec in (("fp64", S.SP_FP64), ("mixed", S.SP_MIXED_BF16X6)):
            plan = S.Plan(p.r_if, p.th_if, p.nphi, precision=prec, tol=1e-10)
            for _ in range(warmup):
                plan.solve(rho, phi)
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                _, info = plan.solve(rho, phi)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1) / steps
            r = {"ms_per_step": ms, "zones_per_s": p.zones / (ms / 1e3), "iterations": info.iterations}
            if ref is not None:
                r["max_rel_err_vs_oracle"] = float(np.max(np.abs(phi.cpu().numpy() - ref)) / np.max(np.abs(ref)))
            res[name] = r
            plan.close()
        out[key] = res
    return out


def run_batched(S, W, torch, dev, check=True, n=64, reps=3):
    """64 independent ragged solves (Nr in [64,512], Ntheta in {32,64,96,128}, Nphi = 2 Ntheta)
    as one sp_solve_batched call; zones/s for float64 and the 6-product mixed mode."""
    probs = W.ragged_batch(n)
    zones = sum(p.zones for p in probs)
    rhos = [torch.from_numpy(p.rho).to(dev) for p in probs]
    out = {"workload": f"ragged_batch: {n} instances, {zones} zones", "instances": n, "zones": zones}
    for name, prec, ragged in (("fp64", S.SP_FP64, False), ("mixed", S.SP_MIXED_BF16X6, False),
                               ("mixed_ragged", S.SP_MIXED_BF16X6, True)):
        S.lib().sp_batched_set_ragged(1 if ragged else 0)
        plans = [S.Plan(p.r_if, p.th_if, p.nphi, precision=prec, tol=1e-10) for p in probs]
        phis = [torch.empty_like(r) for r in rhos]
        S.sp_solve_batched(plans, rhos, phis)          # warm-up (workspaces, module load)
        torch.cuda.synchronize(dev)
        ts = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            infos = S.sp_solve_batched(plans, rhos, phis)
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        launches_ragged = S.lib().sp_batched_last_ragged()
        S.lib().sp_batched_set_ragged(0)
        ms = statistics.median(ts)
        d = {"ms_per_batch": ms, "zones_per_s": zones / (ms / 1e3),
             "form": ("ragged: one launch per step for each of up to 4 groups of instances"
                      if ragged and launches_ragged else "one launch sequence per instance on 8 streams"),
             "max_est_rel_error": max(i.est_rel_error for i in infos),
             "iterations": sorted({int(i.iterations) for i in infos})}
        if check:
            from oracle import sph_poisson as O
            errs = []
            for k in (0, 17, 40):
                q = probs[k]
                ref = O.solve_exact(O.Geometry(q.r_if, q.th_if, q.nphi), q.rho)
                errs.append(float(np.max(np.abs(phis[k].cpu().numpy() - ref)) / np.max(np.abs(ref))))
            d["max_rel_err_vs_oracle_sample"] = max(errs)
        out[name] = d
        for pl in plans:
            pl.close()
    return out


def run_served(S, W, torch, n_requests, rates=(200.0, 2000.0, 20000.0)):
    """Poisson arrivals of solves: 90% one of the 64 ragged-batch instances, 10% the
    550x128x256 workload; 40 GB device-memory budget, resident plans, 8 slots; host
    buffers page-locked as a serving client would keep them.  p50/p99 latency from
    submission to completion, and zones/s."""
    probs = {k: W.ragged_instance(k) for k in range(64)}
    probs[-1] = W.stellar_sh()
    pin = {}
    for k, p in probs.items():
        rho = torch.from_numpy(p.rho).pin_memory().numpy()
        outs = [torch.empty(p.rho.shape, dtype=torch.float64).pin_memory().numpy() for _ in range(4)]
        pin[k] = (rho, outs)
    out = {"workload": f"served_stream: {n_requests} Poisson arrivals, 90% from the 64 ragged-batch instances, "
                       f"10% 550x128x256; 40 GB budget, 8 slots, page-locked host buffers; plans resident and "
                       f"a 200-request burst of the mix served before the measured stream"}
    for name, prec in (("mixed", S.SP_MIXED_BF16X6), ("fp64", S.SP_FP64)):
        for rate in rates:
            if name == "fp64" and rate != rates[0]:
                continue
            srv = S.sp_server_create(40 << 30, 8)
            try:
                for k, p in probs.items():          # make every grid's plan resident (not measured)
                    t, _ = S.sp_server_submit(srv, p.r_if, p.th_if, p.nphi, pin[k][0], pin[k][1][0], precision=prec)
                    S.sp_server_wait(srv, t, 300.0)
                # then a burst of the same mix (not measured): the clones that concurrent
                # requests of one grid need and the slots' grown buffers exist before the
                # measured stream, as in a server that has been running (their allocation
                # time varies with what the GPU's memory held before)
                warm, wuse = [], {k: 0 for k in probs}
                for rq in W.served_stream(200, rate_hz=1e6, seed=11):
                    k = rq["problem"]
                    p = probs[k]
                    buf = pin[k][1][wuse[k] % 4]
                    wuse[k] += 1
                    t, _ = S.sp_server_submit(srv, p.r_if, p.th_if, p.nphi, pin[k][0], buf, precision=prec)
                    warm.append(t)
                for t in warm:
                    S.sp_server_wait(srv, t, 300.0)
                S.sp_server_reset_stats(srv)
                arr = W.served_stream(n_requests, rate_hz=rate, seed=5)
                use = {k: 0 for k in probs}
                tickets = []
                t0 = time.perf_counter()
                for rq in arr:
                    now = time.perf_counter() - t0
                    if rq["t"] > now:
                        time.sleep(rq["t"] - now)
                    k = rq["problem"]
                    p = probs[k]
                    buf = pin[k][1][use[k] % 4]
                    use[k] += 1
                    t, _ = S.sp_server_submit(srv, p.r_if, p.th_if, p.nphi, pin[k][0], buf, precision=prec)
                    tickets.append(t)
                fails = {}
                for t in tickets:
                    st, _ = S.sp_server_wait(srv, t, 300.0)
                    if st != S.SP_OK:
                        fails[S.sp_status_string(st)] = fails.get(S.sp_status_string(st), 0) + 1
                st_ = S.sp_server_stats(srv)
                out[f"{name}@{int(rate)}/s"] = {"p50_ms": st_["p50_ms"], "p99_ms": st_["p99_ms"],
                                                "max_ms": st_["max_ms"], "zones_per_s": st_["zones_per_s"],
                                                "completed": st_["completed"], "failed": fails,
                                                "running_peak": st_["running_peak"],
                                                "evictions": st_["evictions"]}
            finally:
                S.sp_server_destroy(srv)
    return out


# dram__bytes_read.sum + dram__bytes_write.sum per launch, per kernel group, from one ncu
# capture of the mixed solve on the full workload.  The counters hold only for the kernel
# sources they were taken from: `source_sha` is kernel_source_hash() of that build (the
# device code of the mixed path and its launchers), and the bench reports traffic as
# null once those sources differ.
MIXED_KERNEL_SOURCES = ("k_fft.cu", "k_mixed.cu", "fft_dev.cuh", "tc_gemm.cuh", "ff.cuh", "sp_internal.h")
NCU_TRAFFIC = {
    "source_sha": "fe2db1633251d82f",
    "mixed": {   # MB read + written and warp instructions, averaged over the group's launches in one solve
        "fft_forward": {"bytes": (146.65 + 36.54) * 1e6, "inst": 29.28e6, "kernel": "k_fft_fwd<float, double> (rho)"},
        "project_forward": {"bytes": ((91.40 + 18.15) + (91.56 + 18.35)) * 1e6 / 2, "inst": 13.92e6,
                            "kernel": "tc::k_tc_gemm_split<3>"},
        "radial_solve": {"bytes": ((145.83 + 39.07) + (145.80 + 39.12)) * 1e6 / 2, "inst": 19.96e6,
                         "kernel": "k_thomas_scan<2>"},
        "project_inverse": {"bytes": ((91.47 + 18.17) + (91.46 + 18.34)) * 1e6 / 2, "inst": 13.90e6,
                            "kernel": "tc::k_tc_gemm_split<3>"},
        "fft_inverse": {"bytes": ((72.17 + 20.56) + (145.07 + 83.84)) * 1e6 / 2, "inst": (37.17e6 + 56.29e6) / 2,
                        "kernel": "k_fft_inv<float, float, 2> (first solve), k_fft_inv<float, float, 4> (correction)"},
        "residual": {"bytes": (218.82 + 44.18) * 1e6, "inst": 96.09e6,
                     "kernel": "k_residual_fft<0> interior rows (residual and its forward FFT; the last shell, "
                               "0.82 MB and 0.41 M instructions, runs on the side stream)"},
    },
}


def kernel_source_hash(names=MIXED_KERNEL_SOURCES):
    """sha256 (first 16 hex digits) of the named CUDA sources of the library."""
    import hashlib
    h = hashlib.sha256()
    pkg = os.path.join(ROOT, "paper_1806_06623_gb300", "csrc")
    for name in sorted(names):
        h.update(name.encode())
        h.update(open(os.path.join(pkg, name), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(precision, name):
    """Per-launch DRAM bytes of a kernel group from the ncu table, or None when the table
    was taken from other kernel sources (or has no entry)."""
    if NCU_TRAFFIC.get("source_sha") != kernel_source_hash():
        return None
    return NCU_TRAFFIC.get(precision, {}).get(name)


def projection_tensor_rate(timing, p, precision):
    """Tensor-pipe view of the tcgen05 projections: the paper's algorithmic count
    2 Nr Ntheta^2 Nphi flops per projection (Sect. 4.1) and the flops the MMAs execute
    (bf16 products of 128 x 128 x 16 over the padded tiles), per average live launch,
    against the measured dense bf16 burst peak."""
    if precision == "fp64":
        return None
    nr, nth, nphi = p.shape
    mh = nphi // 2 + 1
    ms = sum(timing.get(k, (0.0, 0))[0] for k in ("project_forward", "project_inverse"))
    cnt = sum(timing.get(k, (0.0, 0))[1] for k in ("project_forward", "project_inverse"))
    if not cnt:
        return None
    per_launch_s = ms / cnt / 1e3
    nprod = 6 if precision == "mixed" else 3
    tiles = -(-2 * nr // 128)
    kblocks = -(-nth // 64)
    executed = mh * tiles * kblocks * 4 * nprod * 2.0 * 128 * 128 * 16
    algorithmic = 2.0 * nr * nth * nth * nphi
    try:
        peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"])
        src = "MEASURED_PEAKS.json bf16_tflops (burst, of measured)"
    except Exception:
        peak, src = 1900.0, "fallback 1.9 PFLOP/s"
    a = algorithmic / per_launch_s / 1e12
    e = executed / per_launch_s / 1e12
    return {"us_per_launch": per_launch_s * 1e6, "algorithmic_tflops": a, "algorithmic_frac": a / peak,
            "executed_tflops": e, "executed_frac": e / peak, "peak_tflops": peak, "peak_source": src,
            "products": nprod, "algorithmic": "2 Nr Ntheta^2 Nphi flops per projection",
            "executed": f"{mh} m x {tiles} column tiles x {kblocks} K blocks x 4 x {nprod} MMAs of 128x128x16"}


def algorithmic_bytes_per_step(p, precision, iters=2, fused=None):
    """Bytes each kernel group must move per solve (inputs read once, outputs written once).

    Z = zones, S = spectral values 2 mh Nr Ntheta.  Mixed path with `iters` low-precision
    solves: forward FFTs read rho (8 B) then r (4 B) and write the float32 panel (4 B);
    projections read and write 4 B per spectral value plus the NP bf16 table planes;
    radial solves read the spectrum and both float32 factor tables and write the panel;
    inverse FFTs read the spectrum and write the iterate: the first solve's as its high
    word only (its low word is zero), a correction's reading it and writing both words
    and float64 Phi (the first correction with 6 products float64 Phi only); the residual
    reads rho and the iterate (the high word only after the first solve) and writes r;
    without a correction a separate update reads the high word and writes float64 Phi,
    and with 6 products and a second correction one rebuilds both words from float64.
    Where the library fuses the residual with its forward FFT (`fused`; by default for
    Nphi = 256 and even Ntheta, as the library does) the residual writes the panel (4 B per
    spectral value) instead of r, and the forward FFT group is the transform of rho alone."""
    nr, nth, nphi = p.shape
    mh = nphi // 2 + 1
    Z = float(nr * nth * nphi)
    S = float(2 * mh * nr * nth)
    if precision == "fp64":
        return {"fft_forward": 8 * Z + 8 * S, "project_forward": 16 * S + 8 * mh * nth * nth,
                "radial_solve": 16 * S + 8 * S / 2, "project_inverse": 16 * S + 8 * mh * nth * nth,
                "fft_inverse": 8 * S + 8 * Z}
    npl = 3 if precision == "mixed" else 2
    T = 2.0 * npl * mh * nth * nth
    c = iters - 1   # corrections
    if fused is None:
        fused = nphi == 256 and nth % 2 == 0
    res_out = 4 * S if fused else 4 * Z      # the residual's output: the panel, or r
    return {"fft_forward": (8 * Z + 4 * S) + (0 if fused else c * (4 * Z + 4 * S)),
            "project_forward": iters * (8 * S + T),
            "radial_solve": iters * (4 * S + 4 * S + 4 * S),
            "project_inverse": iters * (8 * S + T),
            "fft_inverse": (4 * S + 4 * Z) + min(c, 1) * (4 * S + (12 if npl == 3 else 20) * Z)
                           + max(c - 1, 0) * (4 * S + 24 * Z),
            "residual": min(c, 1) * (12 * Z + res_out) + max(c - 1, 0) * (16 * Z + res_out),
            "update": 12 * Z if c == 0 else (16 * Z if npl == 3 and c >= 2 else 0.0)}


def roofline(timing, p, precision, steps, iters=2, sm_mhz=None, num_sms=152):
    """Dominant kernel's achieved rate: algorithmic bytes per launch over its average live
    CUDA-event duration (the largest group; for the residual, its interior-row kernel)."""
    nr, nth, nphi = p.shape
    if not timing:
        return None
    # (residual_rows is a span inside the residual's, not a group of its own)
    name, (ms, cnt) = max(((k, v) for k, v in timing.items() if k != "residual_rows"), key=lambda kv: kv[1][0])
    per_launch_s = ms / cnt / 1e3
    share = 1.0
    rows = timing.get("residual_rows", (0.0, 0))
    if name == "residual" and rows[1]:
        # the dominant kernel itself: the residual's interior-row launch, timed on its own
        # stream, and its share (Nr-1)/Nr of the residual's algorithmic bytes; the side
        # stream's shell term and last shell are other kernels
        per_launch_s = rows[0] / rows[1] / 1e3
        share = (nr - 1) / nr
        cnt = rows[1]
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    if name in ("project_forward", "project_inverse") and precision == "fp64":
        flops = 2.0 * nr * nth * nth * nphi            # paper's count per projection (Sect. 4.1)
        ach = flops / per_launch_s / 1e12
        return {"kernel": name, "bound": "alu", "achieved": ach, "peak": 1.25, "unit": "TFLOP/s",
                "frac": ach / 1.25, "traffic": None,
                "peak_source": "nominal GB300 float64 rate (no measured float64 peak on this pool)",
                "algorithmic": "2 Nr Ntheta^2 Nphi flops per projection"}
    per_step = algorithmic_bytes_per_step(p, precision, iters).get(name)
    if per_step is None:
        return None
    b = per_step * steps / cnt * share  # per launch
    ach = b / per_launch_s / 1e9
    pk = float(peaks.get("hbm_gbs", 6800.0))
    tr = ncu_traffic(precision, name)
    label = name if share == 1.0 else "residual_rows (the residual's interior-row kernel)"
    out = {"kernel": label, "bound": "hbm", "achieved": ach, "peak": pk, "unit": "GB/s", "frac": ach / pk,
           "traffic": tr["bytes"] if tr else None, "traffic_kernel": tr["kernel"] if tr else None,
           "algorithmic_bytes_per_launch": b,
           "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6.8 TB/s"}
    if tr and tr.get("inst") and sm_mhz:
        # the instruction-issue view of the same launch: warp instructions (ncu) over the
        # issue rate of 4 per clock per SM at the median SM clock, for the live duration
        issue = 4.0 * num_sms * sm_mhz * 1e6
        out["issue"] = {"warp_instructions_per_launch": tr["inst"], "issue_peak_per_s": issue,
                        "frac": tr["inst"] / (issue * per_launch_s),
                        "peak": f"4 warp instructions per clock per SM x {num_sms} SMs x {sm_mhz:.0f} MHz"}
    return out


def roofline_groups(timing, p, precision, steps, iters=2):
    """Every kernel group's live HBM fraction (algorithmic bytes over its live CUDA-event
    time per step, against the measured copy bandwidth), beside the dominant group's."""
    if not timing or precision == "fp64":
        return None
    try:
        pk = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6800.0))
    except Exception:
        pk = 6800.0
    model = algorithmic_bytes_per_step(p, precision, iters)
    out = {}
    for name, (ms, cnt) in timing.items():
        b = model.get(name)
        if not b or ms <= 0:
            continue
        per_step_s = ms / steps / 1e3
        out[name] = {"ms_per_step": ms / steps, "algorithmic_bytes_per_step": b,
                     "frac": b / per_step_s / 1e9 / pk}
    tot_b = sum(v["algorithmic_bytes_per_step"] for v in out.values())
    tot_s = sum(v["ms_per_step"] for v in out.values()) / 1e3
    out["whole_solve"] = {"ms_per_step": tot_s * 1e3, "algorithmic_bytes_per_step": tot_b,
                          "frac": tot_b / tot_s / 1e9 / pk if tot_s > 0 else None}
    return out


def check_vs_oracle(p, phis):
    """max|dPhi|/max|Phi| against the oracle's exact float64 solution (separated solve
    plus residual correction with the operator) and the backward error eta."""
    from oracle import sph_poisson as O
    geo = O.Geometry(p.r_if, p.th_if, p.nphi)
    ref = O.solve_exact(geo, p.rho)
    out = {}
    for k, v in phis.items():
        if v is None:
            continue
        out[k] = {"max_rel_err": float(np.max(np.abs(v - ref)) / np.max(np.abs(ref))),
                  "eta": O.residuals(geo, v, p.rho)[0]}
    return out


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank)
        return
    run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
