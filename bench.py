"""Benchmark of the active flux hot path (arXiv 2510.11527) on GB300.

Workload (N=1): 2D strongly degenerate Burgers, f = u^2/2 in both directions,
kappa = 0.1 [u > 0.5], discs of +-1 (radius 0.35) on [-1.5, 1.5]^2, 1024^2 periodic
cells, FP64, full MPP limiter + point projection, SSP-RK3. One "step" is one full time
step: the device CFL reduction plus the three fused stage kernels. The metric is
cell-stage updates per second (one cell-stage updates the cell average and the three
point values a cell owns). Synthetic inputs; the L2 cache is flushed between timed
steps and each step is timed with CUDA events on the solver's stream.

Lines printed (rank 0): one JSON object. `--impl reference` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-stage updates/s + HBM roofline fraction, FP32/batched/learned vs plain FP64"
UNIT = "cell-stage updates/s"
FP64_PEAK_TFLOPS = 1.25     # GB300 non-tensor FP64 peak (nominal; a DFMA loop measured 1.19)
# Algorithmic HBM bytes per cell-stage of SSP-RK3 (read the stage input and the RK
# combination input once, write the output once; 10.67 value slots per 4 DoFs).
BYTES_PER_CELL_STAGE = {"fp64": 85.33, "fp32_mixed": 53.33}
# dram__bytes_read.sum + dram__bytes_write.sum per stage launch from the ncu capture
# summarised in profiles/stage2d_fp64_burgers_1024.md (None until captured for this
# kernel version).
NCU_TRAFFIC_PER_LAUNCH = {"fp64": None, "fp32_mixed": None}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_{os.getpid()}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax = float(f[2])
                except ValueError:
                    continue
                for k, nm in enumerate(names):
                    if f[5 + k].lower().startswith("active"):
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def oracle_flops_per_cell(spec, state, tau):
    import oracle
    fc = oracle.flop_count(spec, state, tau)
    return (fc["add"] + fc["mul"] + fc["div"] + fc["exp"]) / spec.cells


def run_gpu(args):
    import torch
    import af_inputs as ai
    from paper_2510_11527_gb300 import Solver, build

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    prec = args.precision
    spec = ai.config2(args.n)
    st = [a.cpu().numpy() for a in ai.initial_state(spec, device="cuda")]
    stream = torch.cuda.Stream()
    solver = Solver(spec, precision=prec, rk=3)
    solver.set_stream(stream)
    solver.set_state(st)
    nst = solver.num_stages
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def one_step():
        solver.dt_device()
        for k in range(nst):
            solver.stage(k, 0.0)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            one_step()
    torch.cuda.synchronize()

    # timed region: per step [dt | stage 0 | stage 1 | stage 2] bracketed by events,
    # L2 flushed between steps (outside the events)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(nst + 2)] for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for s in range(args.steps):
                flush.zero_()
                ev[s][0].record(stream)
                solver.dt_device()
                ev[s][1].record(stream)
                for k in range(nst):
                    solver.stage(k, 0.0)
                    ev[s][2 + k].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    step_ms = [ev[s][0].elapsed_time(ev[s][-1]) for s in range(args.steps)]
    stage_ms = [ev[s][1 + k].elapsed_time(ev[s][2 + k]) for s in range(args.steps) for k in range(nst)]
    dt_ms = [ev[s][0].elapsed_time(ev[s][1]) for s in range(args.steps)]
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    stats = solver.stats()
    lo, hi = solver.bounds()
    cells = spec.cells
    value = world * cells * nst * args.steps / (total_ms / 1e3)

    # end to end through the public API with host buffers: H2D of the step's input,
    # the step, D2H of the result, every step
    e2e_steps = max(2, min(args.steps, 5))
    host = [np.ascontiguousarray(a) for a in st]
    solver.set_state(host)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        solver.set_state(host)
        solver.step(0.0)
        host = solver.get_state()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_value = world * cells * nst * e2e_steps / e2e_s
    bytes_in = sum(a.size * 8 for a in st)

    peaks, peak_src = load_peaks()
    avg_stage_s = statistics.mean(stage_ms) / 1e3
    result = None
    if rank == 0:
        tau = 1e-4
        fpc = oracle_flops_per_cell(ai.config2(256), [a.numpy() for a in ai.initial_state(ai.config2(256))], tau)
        if prec == "fp64":
            ach = fpc * cells / avg_stage_s / 1e12
            roof = {"bound": "alu", "achieved": round(ach, 4), "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": round(ach / FP64_PEAK_TFLOPS, 4), "traffic": NCU_TRAFFIC_PER_LAUNCH[prec],
                    "peak_source": "derived (GB300 FP64 non-tensor nominal)",
                    "flops_per_cell_stage": round(fpc, 1),
                    "hbm_view": {"achieved_gbs": round(BYTES_PER_CELL_STAGE[prec] * cells / avg_stage_s / 1e9, 1),
                                 "peak_gbs": peaks["hbm_gbs"],
                                 "frac": round(BYTES_PER_CELL_STAGE[prec] * cells / avg_stage_s / 1e9 / peaks["hbm_gbs"], 4)}}
        else:
            ach = BYTES_PER_CELL_STAGE[prec] * cells / avg_stage_s / 1e9
            roof = {"bound": "hbm", "achieved": round(ach, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": round(ach / peaks["hbm_gbs"], 4), "traffic": NCU_TRAFFIC_PER_LAUNCH[prec],
                    "peak_source": peak_src}
        result = {
            "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == "fp64" else "f32+f64",
            "data": "synthetic",
            "config": {"workload": f"degenerate_burgers2d_{args.n}x{args.n}_{prec}_ssprk3_mpp",
                       "cells": cells, "stages_per_step": nst, "precision": prec,
                       "l2": "flushed between timed steps (256 MiB write)", "parallelism": f"replicas{world}"},
            "roofline": roof,
            "kernels": {"stage_ms_avg": round(statistics.mean(stage_ms), 5), "dt_reduce_ms_avg": round(statistics.mean(dt_ms), 5)},
            "e2e": {"value": round(e2e_value, 1), "unit": UNIT, "h2d_bytes_per_step": bytes_in,
                    "d2h_bytes_per_step": bytes_in},
            "gpu_launches": (nst + 2) * args.steps,
            "checks": {"bounds": [lo, hi], "safeguard": stats},
            "clocks": clk.summary(),
            "wall_s": round(wall, 3),
        }
    solver.close()
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return result


def cpu_sample(seconds_target=12.0):
    """Time the FP64 oracle on a bounded sample of the workload (config 2 at 512^2)."""
    import af_inputs as ai
    import oracle
    spec = ai.config2(512)
    st = [a.numpy() for a in ai.initial_state(spec)]
    dt = oracle.dt_cfl(spec, st[0])
    t0 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < seconds_target:
        st, _ = oracle.step(spec, 3, st, dt)
        steps += 1
    el = time.perf_counter() - t0
    return {"value": round(spec.cells * 3 * steps / el, 1), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"degenerate_burgers2d 512x512 FP64, {steps} SSP-RK3 steps ({el:.1f} s, single thread)"}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return None
    import af_inputs as ai
    import oracle
    spec = ai.config2(512)
    st = [a.numpy() for a in ai.initial_state(spec)]
    dt = oracle.dt_cfl(spec, st[0])
    for _ in range(args.warmup):
        oracle.step(spec, 3, st, dt)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        st, _ = oracle.step(spec, 3, st, dt)
    el = time.perf_counter() - t0
    value = spec.cells * 3 * args.steps / el
    return {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(el / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "degenerate_burgers2d_512x512_fp64_ssprk3_mpp (bounded sample of the 1024^2 workload)"},
            "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"512x512 cells, {args.steps} SSP-RK3 steps, single thread"},
            "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32_mixed"])
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        res = run_reference(args)
        if res is not None:
            print(json.dumps(res))
        return
    res = run_gpu(args)
    if res is not None:
        rank, world, _ = dist_env()
        if not args.no_cpu_baseline and world == 1:
            res["cpu_baseline"] = cpu_sample()
        print(json.dumps(res))


if __name__ == "__main__":
    main()
