#!/usr/bin/env python
"""RK4-step throughput of the staggered-grid Navier-Stokes solver on one B300 per rank.

Workload: 3-D decaying isotropic turbulence on a 256^3 periodic MAC grid on
[0, 2 pi]^3, nu = 1/1600, seeded random Fourier velocity with
E(k) ~ k^4 exp(-2 (k/4)^2), projected divergence free and scaled to unit
kinetic energy; classic RK4 with a projection every stage and an adaptive
CFL 0.3 time step computed on the device. FP64 and FP32 run side by side;
the headline value is the FP64 one, the FP32 run is reported under "fp32".

A step = one full RK4 step (4 x [F + divergence, FFT Poisson solve,
projection + RK update]) plus the CFL reduction for the next step.
Metric: cell-updates/s = cells * steps / seconds (whole job over all ranks).

Timing: W untimed warm-up steps, then K steps between CUDA events on the
solver's stream, bracketed by a barrier and a device synchronize; the field
(402 MB FP64, 201 MB FP32) is larger than the 126 MB L2, so no L2 flush is
added. Multi-GPU: independent replicas (one trajectory per rank, seed = rank),
no data-path collective; the max time over ranks is used.

--impl reference times the FP64 CPU oracle on this host instead (a bounded
sample: one RK4 step per timed step at 128^3 of the same workload).
"""

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

METRIC = "RK-step cell-updates/s FP64 and FP32 at 256^3 (% of HBM peak); adjoint/forward ratio"
UNIT = "cell-updates/s"
NU = 1.0 / 1600.0
CFL = 0.3


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--dtypes", default="f64,f64n,f32",
                    help="f64: FP64 step (double-float arithmetic where the grid supports it), f64n: FP64 with "
                         "native FP64 arithmetic, f32: FP32")
    ap.add_argument("--no-closure", action="store_true")
    ap.add_argument("--no-channel", action="store_true")
    ap.add_argument("--no-channel-large", action="store_true", help="skip the 512x1024x256 channel point")
    ap.add_argument("--no-wray3", action="store_true")
    ap.add_argument("--no-diff", action="store_true")
    ap.add_argument("--no-les", action="store_true", help="skip the learned-closure training and evaluation")
    ap.add_argument("--sweep", action="store_true", help="FP64 size sweep 128^3..840^3 only (one JSON line)")
    return ap.parse_args()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ byte/op model
# Double-float operations per cell of rhs_div (uniform periodic grid), counted from the kernel's
# source: F^x and F^y 10 additions, 3 products, 11 fused multiply-adds each; F^z 11, 3, 11; D F 3, 1,
# 2; the halo evaluations (one extra F^y per 8 cells, one extra F^x per 32 cells) 1.56, 0.47, 1.72.
# FP32-pipe instructions per double-float operation (results left unnormalised): addition 8 (TwoSum 6 + 2),
# product 4 (TwoProd with fma 2 + 2 fma), fused multiply-add 12.
DF_RHS_OPS = (35.56, 10.47, 36.72)
DF_INST = (8, 4, 12)
DF_RHS_INST = sum(a * b for a, b in zip(DF_RHS_OPS, DF_INST))   # ~767 per cell


def kernel_model(name, n, s, fused=False, arith="native"):
    """Algorithmic bytes and arithmetic per launch of each kernel family.

    N cells, spec = (n/2+1) n^2 complex values of 2 s bytes; s = value size.
    rhs_div: reads u (3N), writes F (3N) and r (N); 79 FP64-pipe ops/cell for F and D F on a
             uniform grid (the count of the kernel as built, with the z-face products of a plane
             carried to the next plane of the march instead of recomputed); in double-float
             arithmetic DF_RHS_INST FP32-pipe instructions per cell.
    update_rhs_div (FP32 fused stage boundary): reads F_s, u_0, acc (9N) and p_s (N), writes acc,
             F_{s+1} (6N) and r (N): 17 values per cell (14 for the first boundary, no acc read).
    fft_*:   each pass reads and writes its data once.
    rk_update: 13 / 16 / 16 / 13 values per cell for stages 1-4 (mean 14.5); only the last stage
             (13) when the stage boundaries are fused.
    """
    N = n ** 3
    spec = (n // 2 + 1) * n * n
    if name == "rhs_div":
        return 7 * N * s, (DF_RHS_INST if arith == "double-float" else 79) * N
    if name == "update_rhs_div":
        return 16 * N * s, None     # stage 1 -> 2 has no accumulator read: (14 + 17 + 17) / 3
    if name == "fft_x_r2c" or name == "fft_x_c2r":
        return N * s + spec * 2 * s, None
    if name == "fft_strided":
        return 2 * spec * 2 * s, None
    if name == "rk_update":
        return (13.0 if fused else 14.5) * N * s, None
    return None, None


# DRAM bytes per launch of the dominant kernels, from ncu captures of the current kernels at n = 256
# (dram__bytes_read.sum + dram__bytes_write.sum of one launch).
TRAFFIC = {("f64n", "rhs_div"): 907.1e6, ("f32", "update_rhs_div"): 1071.0e6,
           ("f64df", "rhs_div"): 913.9e6}   # double-float: mean of stage 1 (916.1 MB) and stages 2-4 (913.2 MB)


def step_model_bytes(n, s):
    """Model bytes of one RK4 step: 114 values per cell (F recomputed in the update; the minimum
    traffic of the scheme: per stage u and F read and written by the fused evaluation and update, the
    Poisson passes over the half spectrum)."""
    return 114 * n ** 3 * s


# ------------------------------------------------------------------ replicas (N > 1)
# The path does not shard (every stencil needs a halo exchange and every Poisson solve all-to-all
# transposes, which the single-GPU design does not do): N processes run independent replicas of the same
# workload (seed + rank), synchronised by barriers around the timed region; the job time is
# the slowest rank's and the throughput counts the cells of all ranks.
def replica_barrier(world):
    import torch.distributed as dist
    if world > 1:
        dist.barrier()


def replica_max(x, world, device):
    """max over ranks of a host float (a one-element tensor on `device` for the collective)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def replica_throughput(cells_per_rank, world, ms_max, steps):
    """Whole-job cell-updates/s: the cells of all ranks over the slowest rank's step time."""
    return cells_per_rank * world / (ms_max / steps / 1e3)


# ------------------------------------------------------------------ our arm
def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2604_18536_b300 import inputs
    from paper_2604_18536_b300.solver import Grid, measure_fma_rate

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (no CPU fallback)")
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        replica_barrier(world)

    def max_over_ranks(x):
        return replica_max(x, world, "cuda")

    n = args.n
    N = n ** 3
    faces = inputs.periodic_box(n, 3)
    raw = inputs.spectrum_velocity_raw(n, 3, seed=args.seed + rank, k0=4.0)
    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs", 6400.0)
    hbm_src = "measured" if "hbm_gbs" in peaks else "fallback"
    fp64_flops = measure_fma_rate(torch.float64)
    fp64_ops_peak = fp64_flops / 2.0          # one FP64 add/mul/fma per pipe slot
    fp32_flops = measure_fma_rate(torch.float32)
    fp32_inst_peak = fp32_flops / 2.0         # FP32 FMA-pipe instructions per second
    results = {}
    for tag in args.dtypes.split(","):
        dtype = torch.float32 if tag == "f32" else torch.float64
        s = 4 if tag == "f32" else 8
        g = Grid(faces, ["periodic"] * 3, NU, dtype=dtype)
        if tag == "f64n":
            g.set_f64_arithmetic("native")
        arith = g.f64_arithmetic() if dtype == torch.float64 else "fp32"
        stream = torch.cuda.current_stream()
        u = torch.tensor(raw, dtype=dtype, device="cuda")
        g.project(u, out=u)
        ke = g.diag(u)["ke"]
        u.mul_(1.0 / math.sqrt(ke))      # unit kinetic energy (initial-condition setup, untimed)
        dt = g.cfl_dt(u, CFL)
        for _ in range(args.warmup):
            g.step(u, dt_dev=dt, next_dt_dev=dt, cfl=CFL)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        clk = ClockSampler(local)
        clk.start()
        time.sleep(0.3)
        # the timed steps: ins_step_n (the steps after the first replay a CUDA graph of one step),
        # no per-kernel events
        l0 = g.launch_count()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.step_n(u, args.steps, dt_dev=dt, next_dt_dev=dt, cfl=CFL)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        launches = g.launch_count() - l0
        clocks = clk.stop()
        barrier()
        ms_max = max_over_ranks(ms)
        # the same K steps as plain ins_step calls (the reference for the adjoint ratio), then once
        # more with a CUDA-event pair around every kernel (per-kernel durations and shares)
        e0.record(stream)
        for _ in range(args.steps):
            g.step(u, dt_dev=dt, next_dt_dev=dt, cfl=CFL)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_plain = max_over_ranks(e0.elapsed_time(e1))
        g.profile(True)
        e0.record(stream)
        for _ in range(args.steps):
            g.step(u, dt_dev=dt, next_dt_dev=dt, cfl=CFL)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_prof = max_over_ranks(e0.elapsed_time(e1))
        prof = g.profile_read()
        g.profile(False)
        diag = g.diag(u)
        # roofline of the dominant kernel (largest share of event-timed time)
        tot = sum(v[1] for v in prof.values())
        dom = max(prof.items(), key=lambda kv: kv[1][1])
        dname, (dl, dms) = dom
        b, ops = kernel_model(dname, n, s, fused=(tag == "f32" and "update_rhs_div" in prof), arith=arith)
        avg_s = dms / dl / 1e3
        traffic = TRAFFIC.get((tag, dname)) if n == 256 else None
        if arith == "double-float" and ops is not None:
            roof = {"bound": "alu", "kernel": dname, "achieved": ops / avg_s / 1e9, "peak": fp32_inst_peak / 1e9,
                    "unit": "G FP32-pipe instructions/s (double-float arithmetic)", "frac": ops / avg_s / fp32_inst_peak,
                    "traffic": TRAFFIC.get(("f64df", dname)) if n == 256 else None,
                    "peak_source": "measured live: dependent FP32 FMA kernel, %.1f TFLOP/s / 2" % (fp32_flops / 1e12),
                    "hbm_frac_of_kernel": (b / avg_s / 1e9) / hbm_peak}
        elif arith == "native" and ops is not None:
            roof = {"bound": "alu", "kernel": dname, "achieved": ops / avg_s / 1e9, "peak": fp64_ops_peak / 1e9,
                    "unit": "Gop/s (FP64 pipe ops)", "frac": ops / avg_s / fp64_ops_peak, "traffic": traffic,
                    "peak_source": "measured live: dependent-FMA kernel, %.3f TFLOP/s / 2" % (fp64_flops / 1e12),
                    "hbm_frac_of_kernel": (b / avg_s / 1e9) / hbm_peak}
        else:
            roof = {"bound": "hbm", "kernel": dname, "achieved": b / avg_s / 1e9, "peak": hbm_peak, "unit": "GB/s",
                    "frac": (b / avg_s / 1e9) / hbm_peak, "traffic": traffic,
                    "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % hbm_src}
        kernels = {k: {"launches": v[0], "total_ms": round(v[1], 4), "share": round(v[1] / tot, 4),
                       "avg_us": round(v[1] / v[0] * 1e3, 2)} for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}
        step_s = ms_max / args.steps / 1e3
        value = replica_throughput(N, world, ms_max, args.steps)
        res = {"value": value, "ms_per_step": ms_max / args.steps, "roofline": roof, "kernels": kernels,
               "ms_per_step_plain_launches": ms_plain / args.steps, "ms_per_step_profiled": ms_prof / args.steps,
               "gpu_launches": launches, "clocks": clocks,
               "step_hbm_frac": step_model_bytes(n, s) / step_s / 1e9 / hbm_peak,
               "final_ke": diag["ke"], "final_max_div": diag["max_div"], "workspace_bytes": g.workspace_bytes(),
               "arithmetic": arith}
        if tag == "f64n":
            # native FP64 arithmetic: the step only (the step VJP and the copies are those of "f64")
            results[tag] = res
            g.close()
            del u
            torch.cuda.empty_cache()
            continue
        # adjoint/forward ratio: ins_step_vjp (stage recompute + reverse sweep) vs ins_step
        kv = max(3, args.steps // 4)
        ybar = u.detach().clone()
        ubar = g.new_velocity()
        nub = torch.zeros(1, dtype=torch.float64, device="cuda")
        g.step_vjp(u, ybar, dt_dev=dt, ubar_n=ubar, nubar=nub)
        torch.cuda.synchronize()
        v0 = torch.cuda.Event(enable_timing=True)
        v1 = torch.cuda.Event(enable_timing=True)
        v0.record(stream)
        for _ in range(kv):
            g.step_vjp(u, ybar, dt_dev=dt, ubar_n=ubar, nubar=nub)
        v1.record(stream)
        torch.cuda.synchronize()
        vms = max_over_ranks(v0.elapsed_time(v1)) / kv
        g.profile(True)
        for _ in range(kv):
            g.step_vjp(u, ybar, dt_dev=dt, ubar_n=ubar, nubar=nub)
        torch.cuda.synchronize()
        vprof = g.profile_read()
        g.profile(False)
        # ratio against the step with the same (plain) launches
        res["adjoint"] = {"ms_per_vjp": vms, "ratio": vms / (ms_plain / args.steps), "vjps": kv,
                          "ratio_vs_graph_step": vms / (ms_max / args.steps),
                          "kernels": {k: {"launches": v[0], "avg_us": round(v[1] / v[0] * 1e3, 2)}
                                      for k, v in sorted(vprof.items(), key=lambda kv_: -kv_[1][1])}}
        del ybar, ubar
        # end to end through the public API with host buffers (pinned), copies inside the timed region
        if not args.no_e2e:
            uh = u.detach().cpu().pin_memory()
            ksteps = max(1, min(args.steps, 5))
            barrier()
            torch.cuda.synchronize()
            f0 = torch.cuda.Event(enable_timing=True)
            f1 = torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            for _ in range(ksteps):
                u.copy_(uh, non_blocking=True)
                g.step(u, dt_dev=dt, next_dt_dev=dt, cfl=CFL)
                uh.copy_(u, non_blocking=True)
            f1.record(stream)
            torch.cuda.synchronize()
            ems = max_over_ranks(f0.elapsed_time(f1))
            res["e2e"] = {"value": N * world / (ems / ksteps / 1e3), "unit": UNIT,
                          "h2d_bytes_per_step": 3 * N * s, "d2h_bytes_per_step": 3 * N * s, "steps": ksteps}
        results[tag] = res
        g.close()
        del u
        torch.cuda.empty_cache()

    if rank == 0:
        prim = results.get("f64") or next(iter(results.values()))
        line = {
            "metric": METRIC, "value": prim["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": prim["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if "f64" in results else "f32",
            "data": "synthetic (seeded random Fourier velocity, E(k)~k^4 exp(-2(k/4)^2), projected, unit KE)",
            "config": {"workload": "3-D decaying isotropic turbulence, 256^3 periodic MAC grid, nu=1/1600, "
                                   "RK4 + per-stage projection, CFL 0.3 (device-side adaptive dt)",
                       "n": n, "cells": N, "global_batch": world, "l2": "inputs larger than L2 (no flush)",
                       "timing": "K steps through ins_step_n (CUDA-graph replay after the first step) between CUDA "
                                 "events; per-kernel durations from a separate pass of K plain steps with an event "
                                 "pair around every kernel",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "ms_per_step_plain_launches": prim["ms_per_step_plain_launches"],
            "ms_per_step_profiled": prim["ms_per_step_profiled"],
            "roofline": prim["roofline"], "e2e": prim.get("e2e"), "gpu_launches": prim["gpu_launches"],
            "clocks": prim["clocks"], "step_hbm_frac": prim["step_hbm_frac"], "kernels": prim["kernels"],
            "adjoint_forward_ratio": prim["adjoint"]["ratio"] if "adjoint" in prim else None,
            "adjoint": prim.get("adjoint"),
            "fp64_arithmetic": prim.get("arithmetic"),
        }
        if "f64n" in results:
            f = results["f64n"]
            line["f64_native"] = {"value": f["value"], "ms_per_step": f["ms_per_step"], "roofline": f["roofline"],
                                  "step_hbm_frac": f["step_hbm_frac"], "kernels": f["kernels"],
                                  "speedup_of_double_float": prim["value"] / f["value"]}
        if "f32" in results and "f64" in results:
            f = results["f32"]
            line["fp32_detail"] = {k: f[k] for k in ("ms_per_step_plain_launches", "ms_per_step_profiled",
                                                      "roofline", "e2e", "gpu_launches", "kernels", "clocks",
                                                      "adjoint", "workspace_bytes") if k in f}
        if not args.no_closure:
            line["closure"] = bench_closure()
        if not args.no_channel:
            line["channel"] = bench_channel()
            if not args.no_channel_large:
                line["channel_large"] = bench_channel_large()
        if not args.no_wray3:
            line["wray3"] = bench_wray3(n, seed=args.seed)
        if not args.no_diff:
            line["differentiation"] = bench_differentiation(seed=args.seed)
        les_res = None
        if not args.no_les and world == 1:
            les_res = bench_les()
            line["closure_les_detail"] = les_res
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline()
        if les_res is not None:
            line["closure_les"] = les_summary(les_res)
        if "f32" in results and "f64" in results:
            # compact FP32 summary as the line's last key (kept short so that a truncated record of the
            # line's tail still carries it)
            f = results["f32"]
            r = f["roofline"]
            line["fp32"] = {"value": f["value"], "ms_per_step": f["ms_per_step"],
                            "step_hbm_frac": round(f["step_hbm_frac"], 4),
                            "speedup_vs_fp64": f["value"] / prim["value"],
                            "step_rel_diff": precision_errors(n, seed=args.seed),
                            "roofline": {"bound": r["bound"], "kernel": r["kernel"], "achieved": round(r["achieved"], 1),
                                         "peak": r["peak"], "unit": r["unit"], "frac": round(r["frac"], 4),
                                         "traffic": r["traffic"]},
                            "e2e": f["e2e"]["value"] if f.get("e2e") else None,
                            "adjoint_forward_ratio": round(f["adjoint"]["ratio"], 3)}
            if "f64n" in results:
                line["fp64_native_ms_per_step"] = results["f64n"]["ms_per_step"]
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


# ------------------------------------------------------------------ size sweep (FP64)
def run_sweep(sizes=(128, 256, 512, 840), steps=5, warmup=2, extra=(("wray3", 840),)):
    """FP64 RK4 step time and device memory at several periodic sizes (one JSON line).

    The initial field is the 3-D Taylor-Green vortex built on the device from separable sines
    (the step's cost does not depend on the field), projected by ins_project."""
    import torch
    from paper_2604_18536_b300 import inputs
    from paper_2604_18536_b300.solver import Grid
    out = []
    for scheme, n in [("rk4", n) for n in sizes] + list(extra):
        torch.cuda.empty_cache()
        free0, total = torch.cuda.mem_get_info()
        g = Grid(inputs.periodic_box(n, 3), ["periodic"] * 3, NU, dtype=torch.float64, scheme=scheme)
        x = (torch.arange(n, dtype=torch.float64, device="cuda") + 0.5) * (2 * math.pi / n)
        xf = (torch.arange(n, dtype=torch.float64, device="cuda") + 1.0) * (2 * math.pi / n)
        u = torch.empty((3, n, n, n), dtype=torch.float64, device="cuda")
        u[0] = torch.sin(xf)[None, None, :] * torch.cos(x)[None, :, None] * torch.cos(x)[:, None, None]
        u[1] = -torch.cos(x)[None, None, :] * torch.sin(xf)[None, :, None] * torch.cos(x)[:, None, None]
        u[2] = 0.0
        g.project(u, out=u)
        dt = g.cfl_dt(u, CFL)
        for _ in range(warmup):
            g.step(u, dt_dev=dt, next_dt_dev=dt, cfl=CFL)
        torch.cuda.synchronize()
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(steps):
            g.step(u, dt_dev=dt, next_dt_dev=dt, cfl=CFL)
        e1.record(st)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        ms = e0.elapsed_time(e1) / steps
        out.append({"n": n, "scheme": scheme, "arithmetic": g.f64_arithmetic(), "ms_per_step": ms,
                    "cell_updates_per_s": n ** 3 / (ms / 1e3),
                    "workspace_gb": g.workspace_bytes() / 1e9, "velocity_gb": u.numel() * 8 / 1e9,
                    "device_used_gb": (free0 - free1) / 1e9})
        g.check_finite()
        g.close()
        del u, x, xf
    print(json.dumps({"sweep": "3-D periodic step (RK4; Wray low-storage RK3 at the end), FP64, CFL 0.3",
                      "results": out}))


# ------------------------------------------------------------------ turbulent channel
def bench_channel(n=(192, 128, 192), steps=10, warmup=3):
    """Re_tau = 180 channel on 4 pi x 2 x 4 pi/3 (tanh y, gamma 1.5), nu = 1/180, f = (1, 0, 0):
    FP64 and FP32 RK4 steps with the device-side CFL 0.3 time step (x/z FFT + FP64 Thomas in y)."""
    import torch
    from paper_2604_18536_b300 import inputs
    from paper_2604_18536_b300.solver import Grid
    faces = inputs.channel_faces(*n)
    raw = inputs.channel_velocity_raw(faces, seed=0)
    out = {"workload": "turbulent channel %dx%dx%d, tanh-stretched y, nu=1/180, RK4, CFL 0.3" % n}
    cells = n[0] * n[1] * n[2]
    for tag, dtype in (("f64", torch.float64), ("f32", torch.float32)):
        g = Grid(faces, ["periodic", "wall", "periodic"], 1.0 / 180, [1.0, 0.0, 0.0], dtype=dtype)
        u = torch.tensor(raw, dtype=dtype, device="cuda")
        g.project(u, out=u)
        dt = g.cfl_dt(u, CFL)
        for _ in range(warmup):
            g.step(u, dt_dev=dt, next_dt_dev=dt, cfl=CFL)
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        # the timed steps as in the main workload: ins_step_n (graph replay after the first step), no
        # per-kernel events; then the same steps as plain calls; then a pass with an event pair around
        # every kernel for the per-kernel durations
        e0.record(st)
        g.step_n(u, steps, dt_dev=dt, next_dt_dev=dt, cfl=CFL)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        e0.record(st)
        for _ in range(steps):
            g.step(u, dt_dev=dt, next_dt_dev=dt, cfl=CFL)
        e1.record(st)
        torch.cuda.synchronize()
        ms_plain = e0.elapsed_time(e1) / steps
        g.profile(True)
        for _ in range(steps):
            g.step(u, dt_dev=dt, next_dt_dev=dt, cfl=CFL)
        torch.cuda.synchronize()
        prof = g.profile_read()
        g.profile(False)
        arith = g.f64_arithmetic() if dtype == torch.float64 else "fp32"
        ms_native = None
        if arith == "double-float":
            # the same steps in native FP64 arithmetic (the step VJP of a wall-bounded grid runs native)
            g.set_f64_arithmetic("native")
            g.step(u, dt_dev=dt, next_dt_dev=dt, cfl=CFL)
            torch.cuda.synchronize()
            e0.record(st)
            for _ in range(steps):
                g.step(u, dt_dev=dt, next_dt_dev=dt, cfl=CFL)
            e1.record(st)
            torch.cuda.synchronize()
            ms_native = e0.elapsed_time(e1) / steps
            g.set_f64_arithmetic("double-float")
        # step VJP on the wall-bounded grid (gather-form transposes, P^T = M Omega P Omega^-1 M)
        ybar = u.detach().clone()
        ubar = g.new_velocity()
        g.step_vjp(u, ybar, dt_dev=dt, ubar_n=ubar)
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(3):
            g.step_vjp(u, ybar, dt_dev=dt, ubar_n=ubar)
        e1.record(st)
        torch.cuda.synchronize()
        vms = e0.elapsed_time(e1) / 3
        g.profile(True)      # per-kernel durations of one more step VJP (a separate pass)
        g.step_vjp(u, ybar, dt_dev=dt, ubar_n=ubar)
        torch.cuda.synchronize()
        vprof = g.profile_read()
        g.profile(False)
        out[tag] = {"ms_per_step": ms, "value": cells / (ms / 1e3), "unit": UNIT, "arithmetic": arith,
                    "ms_per_step_plain_launches": ms_plain,
                    # the channel scheme's minimum traffic: about 110 values per cell and step
                    "step_hbm_frac": 110 * cells * (4 if tag == "f32" else 8) / (ms / 1e3) / 1e9
                    / measured_peaks().get("hbm_gbs", 6400.0),
                    "ms_per_vjp": vms, "adjoint_forward_ratio": vms / ms_plain,
                    "kernels": {k: {"launches": v[0], "avg_us": round(v[1] / v[0] * 1e3, 2)}
                                for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}}
        out[tag]["vjp_kernels"] = {k: {"launches": v[0], "avg_us": round(v[1] / v[0] * 1e3, 2)}
                                   for k, v in sorted(vprof.items(), key=lambda kv: -kv[1][1])}
        if ms_native is not None:
            out[tag]["native_ms_per_step"] = ms_native
            out[tag]["adjoint_forward_ratio_vs_native_step"] = vms / ms_native
            out[tag]["native_note"] = "native FP64: plain ins_step calls"
        g.check_finite()
        g.close()
        del ybar, ubar
    return out


def bench_channel_large(n=(512, 1024, 256), steps=5, warmup=2):
    """Large channel DNS throughput point (the paper's Re_tau = 180 resolution, 512 x 1024 x 256,
    uniform in y): FP64 and FP32 RK4 steps; x/z FFT + FP64 Thomas in y (and the same steps with the
    DCT-II y solve). The initial field (laminar parabola plus sines, projected) is built on the
    device; the step cost does not depend on it."""
    import torch
    from paper_2604_18536_b300 import inputs
    from paper_2604_18536_b300.solver import Grid
    lx, ly, lz = 4 * math.pi, 2.0, 4 * math.pi / 3
    faces = [inputs.uniform_faces(n[0], 0.0, lx), inputs.uniform_faces(n[1], 0.0, ly),
             inputs.uniform_faces(n[2], 0.0, lz)]
    out = {"workload": "channel DNS %dx%dx%d, uniform y, nu=1/180, RK4, CFL 0.3" % n}
    cells = n[0] * n[1] * n[2]
    for tag, dtype in (("f64", torch.float64), ("f32", torch.float32)):
        torch.cuda.empty_cache()
        free0, _ = torch.cuda.mem_get_info()
        g = Grid(faces, ["periodic", "wall", "periodic"], 1.0 / 180, [1.0, 0.0, 0.0], dtype=dtype)
        yc = torch.tensor(inputs.centres(faces[1]), dtype=dtype, device="cuda")
        xf = torch.tensor(faces[0][1:], dtype=dtype, device="cuda")
        zc = torch.tensor(inputs.centres(faces[2]), dtype=dtype, device="cuda")
        env = (yc * (2.0 - yc))[None, :, None]
        u = torch.zeros((3, n[2], n[1], n[0]), dtype=dtype, device="cuda")
        u[0] = 23.4 * env + 1.56 * env * torch.sin(2 * xf)[None, None, :] * torch.cos(3 * zc)[:, None, None]
        u[2] = 1.56 * env * torch.cos(xf)[None, None, :] * torch.sin(2 * zc)[:, None, None]
        g.project(u, out=u)
        dt = g.cfl_dt(u, CFL)
        for _ in range(warmup):
            g.step(u, dt_dev=dt, next_dt_dev=dt, cfl=CFL)
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(steps):
            g.step(u, dt_dev=dt, next_dt_dev=dt, cfl=CFL)
        e1.record(st)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        ms = e0.elapsed_time(e1) / steps
        # the same steps with the DCT-II y solve instead of the Thomas one
        g.set_wall_solver("dct")
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(steps):
            g.step(u, dt_dev=dt, next_dt_dev=dt, cfl=CFL)
        e1.record(st)
        torch.cuda.synchronize()
        ms_dct = e0.elapsed_time(e1) / steps
        out[tag] = {"ms_per_step": ms, "value": cells / (ms / 1e3), "unit": UNIT, "y_solve": "thomas",
                    "dct_ms_per_step": ms_dct, "device_used_gb": (free0 - free1) / 1e9}
        g.check_finite()
        g.close()
        del u, yc, xf, zc, env
        torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------------ low-storage scheme
def bench_wray3(n=256, steps=10, warmup=3, seed=0):
    """Wray's low-storage 3-stage RK on the isotropic-turbulence workload: step and step-VJP
    times, workspace (one velocity register less than RK4)."""
    import torch
    from paper_2604_18536_b300 import inputs
    from paper_2604_18536_b300.solver import Grid
    faces = inputs.periodic_box(n, 3)
    raw = inputs.spectrum_velocity_raw(n, 3, seed=seed, k0=4.0)
    out = {"workload": "3-D decaying isotropic turbulence %d^3, nu=1/1600, Wray low-storage RK3, CFL 0.3" % n}
    for tag, dtype in (("f64", torch.float64), ("f32", torch.float32)):
        g = Grid(faces, ["periodic"] * 3, NU, dtype=dtype, scheme="wray3")
        u = torch.tensor(raw, dtype=dtype, device="cuda")
        g.project(u, out=u)
        u.mul_(1.0 / math.sqrt(g.diag(u)["ke"]))
        dt = g.cfl_dt(u, CFL)
        for _ in range(warmup):
            g.step(u, dt_dev=dt, next_dt_dev=dt, cfl=CFL)
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(steps):
            g.step(u, dt_dev=dt, next_dt_dev=dt, cfl=CFL)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        ybar = u.detach().clone()
        ubar = g.new_velocity()
        g.step_vjp(u, ybar, dt_dev=dt, ubar_n=ubar)
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(3):
            g.step_vjp(u, ybar, dt_dev=dt, ubar_n=ubar)
        e1.record(st)
        torch.cuda.synchronize()
        vms = e0.elapsed_time(e1) / 3
        out[tag] = {"ms_per_step": ms, "value": n ** 3 / (ms / 1e3), "unit": UNIT,
                    "ms_per_vjp": vms, "adjoint_forward_ratio": vms / ms,
                    "workspace_bytes": g.workspace_bytes()}
        g.check_finite()
        g.close()
        del u, ybar, ubar
        torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------------ closure (tensor cores)
def bench_differentiation(n=128, nsteps=16, reps=3, seed=0):
    """Gradient of a 16-step unroll at 128^3 (3-D periodic turbulence, k0 = 4, nu = 1/1000): loss =
    mean squared difference of u_16 to a target 16 steps ahead of the seeded field; torch.autograd over
    ins_step (per-step checkpoints, stage recomputation, ins_step_vjp) for d/du0 and d/dnu. Reports the
    forward unroll time and the forward + backward time per gradient, FP64 and FP32."""
    import torch
    from paper_2604_18536_b300 import inputs
    from paper_2604_18536_b300 import autograd as ag
    from paper_2604_18536_b300.solver import Grid
    out = {"workload": "gradient of a %d-step RK4 unroll, %d^3 periodic, nu=1/1000, w.r.t. u0 and nu" % (nsteps, n)}
    raw = inputs.spectrum_velocity_raw(n, 3, seed=seed, k0=4.0, kmax=n // 4)
    raw1 = inputs.spectrum_velocity_raw(n, 3, seed=seed + 1, k0=4.0, kmax=n // 4)
    for tag, dtype in (("f64", torch.float64), ("f32", torch.float32)):
        g = Grid(inputs.periodic_box(n, 3), ["periodic"] * 3, 1.0 / 1000, dtype=dtype)
        ustar = torch.tensor(raw, dtype=dtype, device="cuda")
        g.project(ustar, out=ustar)
        ustar.mul_(1.0 / math.sqrt(g.diag(ustar)["ke"]))
        pert = torch.tensor(raw1, dtype=dtype, device="cuda")
        g.project(pert, out=pert)
        pert.mul_(0.1 / math.sqrt(g.diag(pert)["ke"]))
        dt = float(g.cfl_dt(ustar, CFL).item())
        target = ustar.clone()
        for _ in range(nsteps):
            g.step(target, dt=dt)
        u0 = ustar + pert

        def grad_once():
            u = u0.detach().clone().requires_grad_(True)
            nut = torch.tensor(g.nu, dtype=torch.float64, device="cuda", requires_grad=True)
            states = ag.rollout(u, g, dt, nsteps, nut)
            loss = ((states[-1] - target) ** 2).mean()
            loss.backward()
            return u.grad, nut.grad

        grad_once()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            with torch.no_grad():
                u = u0.clone()
                for _ in range(nsteps):
                    g.step(u, dt=dt)
        e1.record()
        torch.cuda.synchronize()
        fwd = e0.elapsed_time(e1) / reps
        e0.record()
        for _ in range(reps):
            gu, gnu = grad_once()
        e1.record()
        torch.cuda.synchronize()
        tot = e0.elapsed_time(e1) / reps
        out[tag] = {"ms_forward_unroll": fwd, "ms_per_gradient": tot, "gradient_over_forward": tot / fwd,
                    "backward_over_forward": (tot - fwd) / fwd,
                    "grad_finite": bool(torch.isfinite(gu).all().item() and torch.isfinite(gnu).all().item())}
        g.close()
        del ustar, pert, target, u0
        torch.cuda.empty_cache()
    return out


def precision_errors(n, seed=0):
    """Relative L2 differences of one step from the native-FP64 step of the same (FP32-representable)
    field with the same dt: the FP32 step and the double-float FP64 step, at the benchmark size (the
    native FP64 path itself is within 1e-12 of the FP64 oracle there)."""
    import torch
    from paper_2604_18536_b300 import inputs
    from paper_2604_18536_b300.solver import Grid
    faces = inputs.periodic_box(n, 3)
    g64 = Grid(faces, ["periodic"] * 3, NU, dtype=torch.float64)
    u0 = torch.tensor(inputs.spectrum_velocity_raw(n, 3, seed=seed, k0=4.0), dtype=torch.float64, device="cuda")
    g64.project(u0, out=u0)
    u0.mul_(1.0 / math.sqrt(g64.diag(u0)["ke"]))
    u0 = u0.float().double()
    dt = float(g64.cfl_dt(u0, CFL).item())
    out = {}
    ref = u0.clone()
    supports_df = g64.f64_arithmetic() == "double-float"
    g64.set_f64_arithmetic("native")
    g64.step(ref, dt=dt)
    nrm = torch.linalg.vector_norm(ref)
    if supports_df:
        g64.set_f64_arithmetic("double-float")
        udf = u0.clone()
        g64.step(udf, dt=dt)
        out["double_float_vs_native_fp64"] = float(torch.linalg.vector_norm(udf - ref) / nrm)
        del udf
    g64.close()
    g32 = Grid(faces, ["periodic"] * 3, NU, dtype=torch.float32)
    u32 = u0.float()
    g32.step(u32, dt=dt)
    g32.close()
    out["fp32_vs_native_fp64"] = float(torch.linalg.vector_norm(u32.double() - ref) / nrm)
    del u0, u32, ref
    torch.cuda.empty_cache()
    return out


def bench_les(seeds=64, test=16, nsnap=40, nsteps=10, stride=5, iters=150, batch=8, lr=1e-3):
    """The learned closure end to end at the configured size: filtered DNS from 64 seeded 256^3 FP32
    runs (nu = 1/2000, k0 = 4, 100 spin-up steps, face-averaged to 64^3, nsnap LES steps each), a
    posteriori training of the tensor-core CNN through 10 unrolled LES steps on windows of the 48
    training trajectories (batch 8, Adam lr 1e-3), and per-trajectory spectrum errors of the 16
    held-out trajectories at 10, nsnap/2 and nsnap LES steps, paired against the no-closure LES."""
    from paper_2604_18536_b300 import les
    nu = 1.0 / 2000
    t0 = time.time()
    data = les.dns_dataset(range(seeds), 256, 64, nu, nsnap=nsnap, spinup=100)
    t1 = time.time()
    train_set, test_set = data[:seeds - test], data[seeds - test:]
    windows = les.training_windows(train_set, nsteps, stride)
    W, b, hist = les.train(windows, 64, nu, iters=iters, batch=batch, lr=lr, nsteps=nsteps)
    t2 = time.time()
    horizons = sorted({nsteps, nsnap // 2, nsnap})
    ev = les.evaluate_paired(test_set, 64, nu, W, b, horizons)
    res = {"workload": "learned LES closure: %d filtered 256^3 -> 64^3 DNS trajectories (%d train / %d held out), "
                       "%d LES steps each; training through %d unrolled steps on %d windows, %d Adam iterations"
                       % (seeds, seeds - test, test, nsnap, nsteps, len(windows), iters),
           "final_horizon": nsnap, "loss_first": hist[0], "loss_last": hist[-1], "dns_s": t1 - t0,
           "train_s": t2 - t1, "evaluation": {}}
    for h, r in ev.items():
        res["evaluation"]["H%d" % h] = r
    return res


def les_summary(res):
    """Compact per-horizon summary: means and the paired difference (no closure - closure) +- its SE."""
    out = {}
    for k, r in res["evaluation"].items():
        p = r["closure_vs_no_closure"]
        out[k] = {"no_closure": round(r["no_closure_mean"], 5), "closure": round(r["closure_mean"], 5),
                  "smagorinsky": round(r["smagorinsky_mean"], 5), "paired_diff": round(p["mean_diff"], 5),
                  "se": round(p["se"], 5), "wins": "%d/%d" % (p["wins"], p["n"])}
    return out


def bench_closure(n=64, batch=8, reps=5):
    """CNN closure forward and backward on a training batch of `batch` fields at the LES size n^3 (FP32
    grids, BF16 tensor cores): the batch runs as `batch` calls on one grid, as in training."""
    import torch
    from paper_2604_18536_b300 import inputs
    from paper_2604_18536_b300.closure import Closure, init_params, SHAPES
    from paper_2604_18536_b300.solver import Grid
    g = Grid(inputs.periodic_box(n, 3), ["periodic"] * 3, 1.0 / 2000, dtype=torch.float32)
    c = Closure(g)
    W, b = init_params(0, 1.0)
    c.set_params(W, b)
    us = [torch.tensor(inputs.random_field((3, n, n, n), 1 + i), dtype=torch.float32, device="cuda")
          for i in range(batch)]
    ms = [g.new_velocity() for _ in range(batch)]
    ub = g.new_velocity()
    dW = [torch.zeros_like(w) for w in W]
    db = [torch.zeros_like(x) for x in b]
    c.forward(us[0], ms[0], save=True)
    c.backward(ms[0], ub, dW, db)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]

    def timed(profiled):
        g.profile(profiled)
        fwd = bwd = 0.0
        for _ in range(reps):
            e[0].record(st)
            for i in range(batch):
                c.forward(us[i], ms[i], save=(i == batch - 1))
            e[1].record(st)
            c.backward(ms[batch - 1], ub, dW, db)
            e[2].record(st)
            torch.cuda.synchronize()
            fwd += e[0].elapsed_time(e[1])
            bwd += e[1].elapsed_time(e[2])
        return fwd, bwd

    # batch and backward times as a user sees them (no per-kernel events, which also keep the
    # convolutions' programmatic launches from overlapping), then a pass with an event pair around
    # every kernel for the per-kernel durations
    fwd, bwd = timed(False)
    timed(True)
    prof = g.profile_read()
    g.profile(False)
    c.check()
    N = n ** 3
    flops_fwd = sum(2.0 * N * 27 * ci * co for ci, co in SHAPES)
    conv_ms = sum(v[1] for k, v in prof.items() if k.startswith("conv3d_tc"))
    # conv launches: 4 per forward (batch x reps forwards) + 4 data-gradient launches per backward (reps)
    conv_s = conv_ms / 1e3 / (reps * (batch + 1))
    # the dominant kernel: the 32 -> 32 forward convolutions (two per forward)
    c32 = prof.get("conv3d_tc_32to32", (1, 0.0))
    flops_32 = 2.0 * N * 27 * 32 * 32
    tf_32 = flops_32 / (c32[1] / c32[0] / 1e3) / 1e12 if c32[1] > 0 else 0.0
    peaks = measured_peaks()
    pk = peaks.get("bf16_tflops", 1800.0)
    res = {"n": n, "batch": batch, "fwd_ms_per_batch": fwd / reps, "fwd_ms_per_sample": fwd / reps / batch,
           "bwd_ms_per_sample": bwd / reps, "flops_fwd_per_sample": flops_fwd,
           "fwd_tflops_per_batch": flops_fwd * batch / (fwd / reps / 1e3) / 1e12,
           "conv_tflops": flops_fwd / conv_s / 1e12,
           "roofline": {"bound": "tensor", "kernel": "conv3d_tc (32 -> 32 channels, forward)", "achieved": tf_32,
                        "peak": pk, "unit": "TFLOP/s", "frac": tf_32 / pk, "traffic": None,
                        "flops_per_launch": flops_32,
                        "peak_source": "measured (MEASURED_PEAKS.json bf16_tflops, burst)"},
           "kernels": {k: {"launches": v[0], "avg_us": round(v[1] / v[0] * 1e3, 2)} for k, v in prof.items()}}
    c.close()
    g.close()
    return res


# ------------------------------------------------------------------ oracle on the host
def _oracle_steps(n, steps, warmup, seed):
    """Wall seconds of each of `steps` FP64 oracle RK4 steps (+ CFL) of the workload at n^3, after
    `warmup` untimed steps. Runs in a worker process of the host-core baseline, or in-process."""
    from oracle.grid import Grid as OGrid
    from oracle import poisson, timestep, diagnostics
    from paper_2604_18536_b300 import inputs
    og = OGrid(inputs.periodic_box(n, 3), ["periodic"] * 3, NU)
    u, _ = poisson.project(og, inputs.spectrum_velocity_raw(n, 3, seed=seed, k0=4.0))
    u = u / math.sqrt(diagnostics.kinetic_energy(og, u))
    dt = timestep.cfl_dt(og, u, CFL)
    times = []
    for i in range(warmup + steps):
        t0 = time.perf_counter()
        u = timestep.rk4_step(og, u, dt)
        dt = timestep.cfl_dt(og, u, CFL)
        if i >= warmup:
            times.append(time.perf_counter() - t0)
    return times


def _oracle_worker(args):
    return _oracle_steps(*args)


def host_cpu():
    """(logical cores, CPU model) of this host."""
    model = "unknown"
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return os.cpu_count() or 1, model


def cpu_baseline(n=128, n_big=256, steps=3, warmup=1, seed=0):
    """The FP64 numpy oracle as it stands, timed on the host cores on a bounded sample of the workload.

    The oracle's array arithmetic runs on one thread, so the host cores are used by P independent
    replicas (spawned worker processes, one trajectory each, seed + i) of the n^3 workload: each times
    `steps` RK4 steps after `warmup`; value = sum over replicas of n^3 / (median step time). P is
    bounded by the cores, the free host memory (about 2 GB per 128^3 replica) and 16. The replicas'
    median step time and one step at n_big^3 (the benchmark's size, one process alone) are reported
    beside it."""
    import multiprocessing as mp
    nproc, model = host_cpu()
    try:
        avail = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    except (ValueError, OSError):
        avail = 8e9
    P = max(1, min(nproc, 16, int(avail // 2.5e9)))
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(P) as pool:
        res = pool.map(_oracle_worker, [(n, steps, warmup, seed + i) for i in range(P)])
    wall = time.perf_counter() - t0
    med = [statistics.median(t) for t in res]
    value = sum(n ** 3 / m for m in med)
    t_big = _oracle_steps(n_big, 1, 0, seed)[0]
    return {"value": value, "unit": UNIT, "cores": P, "kind": "oracle",
            "sample": "%d replicas (one process each) of the workload at %d^3, each the median of %d RK4 steps "
                      "after %d warm-up, FP64 numpy oracle (one thread per replica); %.0f s wall"
                      % (P, n, steps, warmup, wall),
            "host": {"nproc": nproc, "cpu_model": model},
            "per_replica_n%d" % n: {"ms_per_step": statistics.median(med) * 1e3,
                                    "note": "median over replicas, measured while all %d ran" % P},
            "n%d_alone" % n_big: {"ms_per_step": t_big * 1e3, "value": n_big ** 3 / t_big, "steps": 1,
                                  "note": "one process, after the replicas finished"}}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n = 128
    from oracle.grid import Grid as OGrid
    from oracle import poisson, timestep, diagnostics
    from paper_2604_18536_b300 import inputs
    faces = inputs.periodic_box(n, 3)
    og = OGrid(faces, ["periodic"] * 3, NU)
    u, _ = poisson.project(og, inputs.spectrum_velocity_raw(n, 3, seed=args.seed, k0=4.0))
    u = u / math.sqrt(diagnostics.kinetic_energy(og, u))
    dt = timestep.cfl_dt(og, u, CFL)
    for _ in range(args.warmup):
        u = timestep.rk4_step(og, u, dt)
        dt = timestep.cfl_dt(og, u, CFL)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        u = timestep.rk4_step(og, u, dt)
        dt = timestep.cfl_dt(og, u, CFL)
    sec = time.perf_counter() - t0
    value = n ** 3 * args.steps / sec
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded random Fourier velocity)",
            "config": {"workload": "3-D decaying isotropic turbulence, nu=1/1600, RK4 + per-stage projection, "
                                   "CFL 0.3; bounded CPU sample at 128^3 of the 256^3 workload", "n": n},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "%d RK4 steps at 128^3, FP64 numpy oracle" % args.steps},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse()
    if args.sweep:
        run_sweep()
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
