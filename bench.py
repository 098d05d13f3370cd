#!/usr/bin/env python
"""CTMRG sweeps/s on one GB300 (per GPU; N GPUs run independent replicas).

Workload (default): S=1 spins d=3, D=8, chi=128 (N = chi D^2 = 8192), 2x2
cell, x-polarised product state + 0.05 N(0,1) (seed 3), random environment
(seed 4).  One step = one full CTMRG sweep (left, top, right, bottom moves:
64 enlarged corners, 16 projectors by randomised SVD, 16 site updates).

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOADS = {
    "xpol_d3_D8_chi128": "d=3 (S=1), D=8, chi=128, 2x2 cell, x-polarised + 0.05 noise (seed 3), env seed 4",
    "neel_d2_D6_chi72": "d=2, D=6, chi=72, 2x2 cell, Neel + 0.1 noise (seed 2), env seed 3",
    "neel_d2_D3_chi16": "d=2, D=3, chi=16, 2x2 cell, Neel + 0.1 noise (seed 0), env seed 1",
}
METRIC = "CTMRG sweeps/s at D=8,chi=128 (d=3, 2x2 cell)"
FP64_NOMINAL_TFLOPS = 1.25  # GB300 FP64 (profiling recipe, nominal)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--slices", type=int, default=5)
    ap.add_argument("--workload", default="xpol_d3_D8_chi128", choices=sorted(WORKLOADS))
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def max_over_ranks(x, world, device):
    """Largest x over all ranks: a replicated job takes as long as its
    slowest rank."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank, world, seconds_max):
    """Whole-job throughput of `world` independent replicas, timed by the slowest."""
    return world * units_per_rank / seconds_max


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx = float(r[1])
                for n, v in zip(names, r[4:8]):
                    if v.lower() in ("active", "1"):
                        reasons.add(n)
            except (ValueError, IndexError):
                pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle: bounded sample = one cut's projectors (4 enlarged corners,
# dense half systems, M = H_u^T H_d, full SVD); a sweep has 16 cuts.
# ---------------------------------------------------------------------------
def oracle_cut_seconds(workload):
    from oracle import ctmrg_ref as R
    from paper_2112_13184_gb300 import inputs as I
    w = I.workload(workload)
    t = time.perf_counter()
    Qs = R.cut_corners(w["envs"], w["As"], 0, 0, 2, 2)
    R.projectors(*Qs, w["chi"])
    return time.perf_counter() - t


def oracle_corner_seconds(workload):
    """A short oracle sample: one enlarged corner of site 0 (warm-up steps of
    the reference arm; NumPy has no warm-up state to build)."""
    from oracle import ctmrg_ref as R
    from paper_2112_13184_gb300 import inputs as I
    w = I.workload(workload)
    e = w["envs"][0]
    t = time.perf_counter()
    R.enlarged_ul(e["C1"], e["T1"], e["T4"], w["As"][0])
    return time.perf_counter() - t


def cpu_baseline(workload, reps=1):
    ts = [oracle_cut_seconds(workload) for _ in range(reps)]
    t = min(ts)
    return {"value": 1.0 / (16.0 * t), "unit": "sweeps/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"one cut's projectors of {workload} (4 enlarged corners, dense H_u, H_d, "
                      f"M = H_u^T H_d, full LAPACK SVD) = 1/16 of a sweep, {t:.1f} s; the absorption "
                      "step is not timed (it is cheaper than the projector)"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_corner_seconds(args.workload)
    ts = [oracle_cut_seconds(args.workload) for _ in range(args.steps)]
    total = sum(ts)
    value = args.steps / (16.0 * total)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "sweeps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 16.0 * total / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "desc": WORKLOADS[args.workload]},
            "cpu_baseline": {"value": value, "unit": "sweeps/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": "each timed step: one cut's projectors (4 enlarged corners, dense H_u, H_d, "
                                       "M, full LAPACK SVD) = 1/16 sweep of the workload; each warm-up "
                                       "step: one enlarged corner"},
            "e2e": {"value": value, "unit": "sweeps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def oz_gemm_roofline(by_op):
    """Roofline of the emulated-FP64 GEMM class (k_oz_gemm) over one sweep.

    Each operation tag records its tensor flops (2 M N K per BF16 slice
    product, s(s+1)/2 products) and algorithmic bytes (BF16 slices of both
    operands + FP64 output).  Per tag the roofline time is
    max(F / P_tensor, B / BW); the class is reported in the unit of the
    bound that dominates its summed roofline time, with the roofline-time
    fraction (sum of roofline times / measured time) beside it."""
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    tc = peaks["bf16_tflops_sustained"] * 1e12
    bw = peaks["hbm_gbs"] * 1e9
    F = B = T = t_tc = t_bw = t_roof = 0.0
    ops = {}
    for tag, v in by_op.items():
        if not tag.endswith("/gemm") or v["ms"] <= 0:
            continue
        f, b, t = v["flops"], v["bytes"], v["ms"] / 1e3
        tr = max(f / tc, b / bw)
        F, B, T = F + f, B + b, T + t
        t_tc, t_bw, t_roof = t_tc + f / tc, t_bw + b / bw, t_roof + tr
        ops[tag] = {"ms": round(v["ms"], 3), "bound": "tensor" if f / tc >= b / bw else "hbm",
                    "roofline_frac": round(tr / t, 4)}
    if T <= 0:
        return None
    tensor = t_tc >= t_bw
    achieved = F / T / 1e12 if tensor else B / T / 1e9
    peak = tc / 1e12 if tensor else bw / 1e9
    top = dict(sorted(ops.items(), key=lambda kv: -kv[1]["ms"])[:8])
    return {"bound": "tensor" if tensor else "hbm", "kernel": "k_oz_gemm (tcgen05 BF16 slice products)",
            "achieved": achieved, "peak": peak, "unit": "TFLOP/s" if tensor else "GB/s",
            "frac": achieved / peak, "traffic": None,
            "peak_source": ("MEASURED_PEAKS.json bf16_tflops_sustained (of measured)" if tensor
                            else "MEASURED_PEAKS.json hbm_gbs (of measured)"),
            "roofline_time_frac": t_roof / T, "class_ms": T * 1e3,
            "note": ("achieved = sum over the sweep's emulated GEMMs of the algorithmic work in the "
                     "bound's unit / their summed device time; roofline_time_frac = "
                     "sum max(F/P_tensor, B/BW) / measured time (shapes range from tensor- to "
                     "HBM-bound); traffic: per-shape DRAM bytes are in profiles/"),
            "ops": top}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2112_13184_gb300 import ctm as C
    from paper_2112_13184_gb300 import inputs as I

    w = I.workload(args.workload)
    d, D, chi = w["d"], w["D"], w["chi"]
    prec = C.CTM_OZAKI_BF16 if args.precision == "mixed" else C.CTM_FP64
    stream = torch.cuda.Stream()
    solver = C.CTMRG(d, D, chi, stream=stream, precision=prec, seed=rank, ozaki_slices=args.slices)
    solver.set_tensors(w["As"])
    solver.set_envs(w["envs"])

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()

    # warm-up (the first sweep is eager; warm sweeps replay one CUDA graph)
    solver.sweep(args.warmup)
    # timed: K sweeps on the handle's stream, inputs resident in HBM
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.nvtx.range_push("timed")  # lets a profiler keep to the timed sweeps
        ev0.record(stream)
        solver.sweep(args.steps)
        ev1.record(stream)
        barrier()
        torch.cuda.nvtx.range_pop()
    ms = ev0.elapsed_time(ev1)
    # kernels launched per sweep: counted on one eager, event-timed sweep
    # (graph replays launch the same kernels without host calls); the same
    # sweep gives the per-class device times for the roofline
    C.ctm_profile_enable(solver.h, True)
    C.ctm_profile_read(solver.h, reset=True)
    l0 = C.ctm_kernel_launches()
    solver.sweep(1)
    launches = (C.ctm_kernel_launches() - l0) * args.steps
    by_op = C.ctm_profile_report(solver.h)
    prof = C.ctm_profile_read(solver.h, reset=True)
    C.ctm_profile_enable(solver.h, False)
    ms_max = max_over_ranks(ms, world, "cuda")
    value = replica_throughput(args.steps, world, ms_max / 1e3)

    # end to end through the C ABI with host buffers: per step copy A and the
    # environment in from pinned host memory, one sweep, environment out
    pin_A = [torch.from_numpy(a).pin_memory() for a in w["As"]]
    envs_h = solver.get_envs()
    pin_env = [{k: torch.from_numpy(v).pin_memory() for k, v in e.items()} for e in envs_h]
    h2d = sum(a.numel() * 8 for a in pin_A) + sum(v.numel() * 8 for e in pin_env for v in e.values())
    d2h = sum(v.numel() * 8 for e in pin_env for v in e.values())
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        for i, a in enumerate(pin_A):
            C.ctm_set_tensor(solver.h, i, a.numpy())
        for i, e in enumerate(pin_env):
            for k, v in e.items():
                C.ctm_set_env(solver.h, i, k, v.numpy())
        solver.sweep(1)
        for i, e in enumerate(pin_env):
            for k, v in e.items():
                v.copy_(torch.from_numpy(C.ctm_get_env(solver.h, i, k, tuple(v.shape))))
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_max = max_over_ranks(e2e_s, world, "cuda")
    e2e_value = replica_throughput(args.e2e_steps, world, e2e_max) if args.e2e_steps > 0 else None

    if rank == 0:
        g = prof["gemm"]
        achieved = g["flops"] / (g["ms"] / 1e3) / 1e12 if g["ms"] > 0 else None
        prof_note = ("per-class device time of one eager sweep with CUDA events around every call, "
                     "run right after the timed region (graph replays cannot be timed per kernel)")
        if prec == C.CTM_FP64:
            roof = {"bound": "alu", "kernel": "k_dgemm (FP64 DFMA)", "achieved": achieved,
                    "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP64_NOMINAL_TFLOPS if achieved else None, "traffic": None,
                    "peak_source": "GB300 FP64 nominal 1.25 TFLOP/s (profiling recipe table)"}
        else:
            roof = oz_gemm_roofline(by_op)
        total_ms = sum(p["ms"] for p in prof.values())
        line = {
            "metric": METRIC, "value": value, "unit": "sweeps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == C.CTM_FP64 else "bf16x-slices->f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "desc": WORKLOADS[args.workload], "precision": args.precision,
                       "slices": args.slices if prec != C.CTM_FP64 else None,
                       "parallelism": f"replicas x{world}",
                       "l2": "working set per sweep (N x N corners, 537 MB each) exceeds the 129 MB L2"},
            "roofline": roof,
            "e2e": {"value": e2e_value, "unit": "sweeps/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "steps": args.e2e_steps},
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "profile_note": prof_note,
            "profile_by_op": {k: {"ms": round(v["ms"], 3), "calls": v["calls"], "launches": v.get("launches")}
                              for k, v in sorted(by_op.items(), key=lambda kv: -kv[1]["ms"])},
            "profile": {k: {"ms": round(v["ms"], 3), "share": round(v["ms"] / total_ms, 4) if total_ms else None,
                            "calls": v["calls"], "tflops": (v["flops"] / (v["ms"] / 1e3) / 1e12)
                            if v["ms"] > 0 and v["flops"] > 0 else None}
                        for k, v in prof.items()},
        }
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args.workload)
        print(json.dumps(line), flush=True)
    solver.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
