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
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-stage updates/s + HBM roofline fraction, FP32/batched/learned vs plain FP64"
UNIT = "cell-stage updates/s"
FP64_PEAK_TFLOPS = 1.25     # GB300 non-tensor FP64 peak (nominal; a DFMA loop measured 1.19)
# Algorithmic FP64 flops of one limited forward-Euler evaluation per cell on the
# degenerate Burgers workload (adds, multiplies, divisions and exponentials counted by
# the oracle's counting scalar on the 256^2 case; tests/test_bench_constants.py
# recomputes it).
FLOPS_PER_CELL_STAGE = 571.03
# Algorithmic HBM bytes per cell-stage of SSP-RK3 (read the stage input and the RK
# combination input once, write the output once; 10.67 value slots per 4 DoFs).
BYTES_PER_CELL_STAGE = {"fp64": 85.33, "fp32_mixed": 53.33}
# SSP-RK(5,4) in the stage layout of the library: 2 + 3 + 3 + 5 + 3 = 16 state passes
# over 5 stages (the fourth stage reads U3, U0, U2 and writes U1, U2), 3.2 per stage.
BYTES_PER_CELL_STAGE_RK54 = {"fp64": 102.4, "fp32_mixed": 64.0}
# 1D interval with Dirichlet ends (Example 6.5): algorithmic flops of one limited
# forward-Euler evaluation per cell (oracle count on its initial data at 65536 cells) for
# the doubly conservative form and the form without double conservation, and the bytes
# a stage must move per cell (SSP-RK3: (2 + 3 + 3) / 3 passes over ub and one point
# value per cell).
FLOPS_PER_CELL_STAGE_1D = {"dc": 135.12, "nodc": 209.05}
BYTES_PER_CELL_STAGE_1D = {"fp64": 42.67, "fp32_mixed": 32.0}
# 3D (8 FP64 arrays per state): SSP-RK3 passes (2 + 3 + 3) / 3 per stage; and the
# algorithmic flops of one limited forward-Euler evaluation per cell on the 3D
# porous-medium workload (the oracle's count, pointwise functions evaluated once per
# location as in the 2D count; f = 0, whose convection terms neither side forms)
BYTES_PER_CELL_STAGE_3D = 170.67
FLOPS_PER_CELL_STAGE_3D = 791.56
# dram__bytes_read.sum + dram__bytes_write.sum of one stage launch (SSP-RK3 stage 2) from
# the ncu captures summarised in profiles/stage2d_fp64_degenerate_burgers_1024.md and
# profiles/stream2d_fp32mixed_degenerate_burgers_2048.md, keyed by (precision, n); null
# for any other size.
NCU_TRAFFIC_PER_LAUNCH = {("fp64", 1024): 74.79e6, ("fp32_mixed", 2048): 229.67e6}
# thread instructions per cell-stage of the FP32-mixed (column-marching) stage from the
# same capture (smsp__inst_executed.sum x 32 / cells)
NCU_INSTR_PER_CELL_STAGE = {("fp32_mixed", 2048): 769.0}


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
        fd, self.path = tempfile.mkstemp(prefix="af_clocks_", suffix=".csv")
        os.close(fd)

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.fh,
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


def max_over_ranks(value, device="cpu"):
    """Maximum of a per-rank float over all ranks (the bench's timing rule); identity
    without an initialised process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


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
    bl = args.workload == "buckley_leverett_plain_blend"
    if bl and prec != "fp32_mixed":
        raise SystemExit("the Buckley-Leverett blend workload is timed in fp32_mixed only")
    spec = ai.config5(args.n) if bl else ai.config2(args.n)
    st = [a.cpu().numpy() for a in ai.initial_state(spec, device="cuda")]
    wname = (f"buckley_leverett2d_{args.n}x{args.n}_{prec}_ssprk3_mpp_plain_blend" if bl else
             f"degenerate_burgers2d_{args.n}x{args.n}_{prec}_ssprk3_mpp")
    tkey = ("bl_blend" if bl else "") + prec
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
    total_ms = max_over_ranks(sum(step_ms), device="cuda")
    stats = solver.stats()
    lo, hi = solver.bounds()
    cells = spec.cells
    value = world * cells * nst * args.steps / (total_ms / 1e3)

    # end to end through the public API with host buffers: H2D of the step's input,
    # the step, D2H of the result, every step
    # (pinned host buffers; each step's result is the next step's input)
    e2e_steps = max(2, min(args.steps, 20))
    pin_in = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in st]
    pin_out = [torch.empty(a.shape, dtype=torch.float64).pin_memory() for a in st]
    host_in, host_out = [t.numpy() for t in pin_in], [t.numpy() for t in pin_out]
    solver.set_state(host_in)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        solver.set_state(host_in)
        solver.step(0.0)
        solver.get_state(out=host_out)
        host_in, host_out = host_out, host_in
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_value = world * cells * nst * e2e_steps / e2e_s
    bytes_in = sum(a.size * 8 for a in st)

    peaks, peak_src = load_peaks()
    avg_stage_s = statistics.mean(stage_ms) / 1e3
    result = None
    if rank == 0:
        fpc = FLOPS_PER_CELL_STAGE
        if prec == "fp64":
            ach = fpc * cells / avg_stage_s / 1e12
            roof = {"bound": "alu", "achieved": round(ach, 4), "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": round(ach / FP64_PEAK_TFLOPS, 4), "traffic": NCU_TRAFFIC_PER_LAUNCH.get((tkey, args.n)),
                    "peak_source": "derived (GB300 FP64 non-tensor nominal)",
                    "flops_per_cell_stage": round(fpc, 1),
                    "hbm_view": {"achieved_gbs": round(BYTES_PER_CELL_STAGE[prec] * cells / avg_stage_s / 1e9, 1),
                                 "peak_gbs": peaks["hbm_gbs"],
                                 "frac": round(BYTES_PER_CELL_STAGE[prec] * cells / avg_stage_s / 1e9 / peaks["hbm_gbs"], 4)}}
        else:
            ach = BYTES_PER_CELL_STAGE[prec] * cells / avg_stage_s / 1e9
            roof = {"bound": "hbm", "achieved": round(ach, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": round(ach / peaks["hbm_gbs"], 4), "traffic": NCU_TRAFFIC_PER_LAUNCH.get((tkey, args.n)),
                    "peak_source": peak_src}
            ipc = NCU_INSTR_PER_CELL_STAGE.get((tkey, args.n))
            if ipc:
                # what actually bounds this form: instruction issue (one warp instruction
                # per clock per SM sub-partition at the sampled maximum SM clock)
                props = torch.cuda.get_device_properties(local)
                mhz = clk.summary().get("sm_max_mhz") or 2070.0
                peak_issue = props.multi_processor_count * 4 * mhz * 1e6
                got = ipc / 32 * cells / avg_stage_s
                roof["issue_view"] = {"warp_instr_per_cell_stage": round(ipc / 32, 2), "achieved": round(got, 1),
                                      "peak": round(peak_issue, 1), "unit": "warp instructions/s",
                                      "frac": round(got / peak_issue, 4)}
        result = {
            "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == "fp64" else "f32+f64",
            "data": "synthetic",
            "config": {"workload": wname,
                       "cells": cells, "stages_per_step": nst, "precision": prec,
                       "l2": "flushed between timed steps (256 MiB write)", "parallelism": f"replicas{world}"},
            "roofline": roof,
            "kernels": {"stage_ms_avg": round(statistics.mean(stage_ms), 5), "dt_reduce_ms_avg": round(statistics.mean(dt_ms), 5)},
            "e2e": {"value": round(e2e_value, 1), "unit": UNIT, "h2d_bytes_per_step": bytes_in,
                    "d2h_bytes_per_step": bytes_in},
            # per step: the CFL rate and its finalisation, one stage launch per stage (and
            # the plain indicator's pass before each blended stage)
            "gpu_launches": (nst * (2 if bl else 1) + 2) * args.steps,
            "checks": {"bounds": [lo, hi], "safeguard": stats},
            "clocks": clk.summary(),
            "wall_s": round(wall, 3),
        }
    solver.close()
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return result


# ---------------------------------------------------------------------------------------
# the other forms of the metric: FP32-mixed, batched, learned (each against plain FP64)

def _cuda_view(ptr, shape, typestr):
    import torch

    class _V:
        __cuda_array_interface__ = {"shape": shape, "typestr": typestr, "data": (ptr, False), "version": 3}

    return torch.as_tensor(_V(), device="cuda")


def _load_device(solver, state_dev):
    """Copy a device state (FP64 tensors) into the solver's buffers without a host trip."""
    import torch
    for dst, src in zip(solver.device_tensors(), state_dev):
        dst.copy_(src.to(dst.dtype))
    torch.cuda.synchronize()   # the solver runs on its own stream


def _time_steps(stepper, nst, steps, warmup, stream, flush=None):
    """CUDA-event timing of `steps` steps on `stream`: returns (step_ms, stage_ms)."""
    import torch
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            stepper(None)
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(nst + 2)] for _ in range(steps)]
    with torch.cuda.stream(stream):
        for s in range(steps):
            if flush is not None:
                flush.zero_()
            stepper(evs[s])
    torch.cuda.synchronize()
    step_ms = [e[0].elapsed_time(e[-1]) for e in evs]
    stage_ms = [e[1 + k].elapsed_time(e[2 + k]) for e in evs for k in range(nst)]
    return step_ms, stage_ms


def _solver_stepper(solver, stream):
    nst = solver.num_stages

    def step(ev):
        if ev:
            ev[0].record(stream)
        solver.dt_device()
        if ev:
            ev[1].record(stream)
        for k in range(nst):
            solver.stage(k, 0.0)
            if ev:
                ev[2 + k].record(stream)
    return step


def _single_form(spec, prec, steps, warmup, state_dev, stream, flush=None, net=None, rk=3):
    import statistics as st_
    from paper_2510_11527_gb300 import Solver, capi
    s = Solver(spec, precision=prec, rk=rk)
    s.set_stream(stream)
    # bounds and a valid initial state are set through the API on a 1x copy, then the
    # full device state is written in place
    _load_device(s, state_dev)
    if net is not None:
        capi.af_set_mlp(s.ctx, net)
    step_ms, stage_ms = _time_steps(_solver_stepper(s, stream), s.num_stages + (0), steps, warmup, stream, flush)
    out = {"value": spec.cells * s.num_stages * steps / (sum(step_ms) / 1e3), "ms_per_step": st_.mean(step_ms),
           "stage_ms_avg": st_.mean(stage_ms), "stats": s.stats()}
    return s, out


def _hbm_roof(prec, cells, stage_ms, peaks, extra_bytes=0.0, rk=3):
    b = (BYTES_PER_CELL_STAGE if rk == 3 else BYTES_PER_CELL_STAGE_RK54)[prec] + extra_bytes
    ach = b * cells / (stage_ms / 1e3) / 1e9
    return {"bound": "hbm", "achieved": round(ach, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": round(ach / peaks["hbm_gbs"], 4), "bytes_per_cell_stage": b}


def forms(args, headline_value, peaks):
    """FP32-mixed, batched and learned forms of the metric, each with its speedup over
    the plain FP64 GPU form on the same workload and its L1 difference from FP64."""
    import torch
    stream = torch.cuda.Stream()
    res = {}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    sel = set(args.forms.split(","))
    if "fp32" in sel:
        res.update(_form_fp32(args, stream, flush, peaks))
    if "rk54" in sel:
        res.update(_form_rk54(args, stream, flush, peaks))
    if "pme" in sel:
        res.update(_form_pme(args, stream, peaks))
    if "batch" in sel:
        res.update(_form_batch(args, stream, headline_value, peaks))
    if "bl" in sel:
        res.update(_form_bl(args, stream, peaks))
    if "bounded1d" in sel:
        res.update(_form_bounded1d(args, stream, peaks))
    if "ex65" in sel:
        res.update(_form_ex65())
    if "ex64_66" in sel:
        res.update(_form_examples_64_66())
    if "rect2d" in sel:
        res.update(_form_rect2d(args, stream, flush, peaks))
    if "pme3d" in sel:
        res.update(_form_pme3d(args, stream, peaks))
    if "pme_full" in sel:
        res.update(_form_pme_full(args))
    if "c2_full" in sel:
        res.update(_form_c2_full(args))
    return res


def _form_pme_full(args):
    """The porous-medium workload run to its final time: Barenblatt profile (m = 2) at
    t = 1 on [-10, 10]^2, to t = 2, SSP-RK(5,4) at the default (capped) step.
    FP32-mixed at --pme-n cells per direction and both forms at 1024^2: time to
    solution, steps, L1 / Linf of the cell averages against the closed form's averages,
    FP32-mixed against FP64 on the same mesh, bounds, mass change and safeguard clamps."""
    import math
    import time
    import torch
    import af_inputs as ai
    from paper_2510_11527_gb300 import Solver
    out = {}
    finals = {}
    for n, prec in ((1024, "fp64"), (1024, "fp32_mixed"), (args.pme_n, "fp32_mixed")):
        key = (n, prec)
        if key in finals:
            continue
        spec = ai.config3(n)
        st = [a.cpu().numpy() for a in ai.state_2d(lambda x, y: ai.barenblatt(x, y, 1.0), spec, device="cuda", sub=2,
                                                    order=3)]
        exact = ai.state_2d(lambda x, y: ai.barenblatt(x, y, 2.0), spec, device="cuda", sub=2, order=3)[0]
        with Solver(spec, precision=prec, rk=54) as s:
            s.set_state(st)
            m0 = s.mass()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            steps = s.run(1.0)
            torch.cuda.synchronize()
            secs = time.perf_counter() - t0
            ub = torch.from_numpy(s.get_state()[0]).cuda().reshape(exact.shape)
            lo, hi = s.bounds()
            stats = s.stats()
            m1 = s.mass()
        d = (ub - exact).abs()
        finals[key] = ub
        out[f"pme_t2_{prec}_{n}"] = {
            "steps": steps, "seconds": round(secs, 2), "cell_stage_per_s": round(spec.cells * 5 * steps / secs, 1),
            "l1_vs_closed_form": float(d.mean()), "linf_vs_closed_form": float(d.max()), "min": lo, "max": hi,
            "mass_rel_change": (m1 - m0) / m0, "clamps": stats["clamps"], "errors": stats["errors"]}
        del exact, ub
    a, b = finals[(1024, "fp32_mixed")], finals[(1024, "fp64")]
    out["pme_t2_fp32_vs_fp64_1024"] = {"l1": float((a - b).abs().mean()), "linf": float((a - b).abs().max())}
    return out


def _form_c2_full(args):
    """The degenerate Burgers workload (1024^2) run to its final time T = 0.5 with
    SSP-RK3 at the default step, FP32-mixed (and FP64 with --c2-fp64): steps, time to
    solution, bounds, the safeguard's counts (values clamped, of which cell averages;
    the largest excess) and the relative mass change; with FP64, the L1
    / Linf distance of the FP32-mixed cell averages to FP64's."""
    import time
    import numpy as np
    import torch
    import af_inputs as ai
    from paper_2510_11527_gb300 import Solver
    spec = ai.config2(1024)
    st = [a.cpu().numpy() for a in ai.initial_state(spec, device="cuda")]
    scale = float(np.sum(np.abs(st[0]))) * spec.dx * spec.dy
    out, finals = {}, {}
    for prec in (("fp32_mixed", "fp64") if args.c2_fp64 else ("fp32_mixed",)):
        with Solver(spec, precision=prec) as s:
            s.set_state(st)
            m0 = s.mass()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            steps = s.run(0.5)
            torch.cuda.synchronize()
            secs = time.perf_counter() - t0
            finals[prec] = s.get_state()[0]
            lo, hi = s.bounds()
            stats = s.stats()
            m1 = s.mass()
        out[f"config2_T05_{prec}_1024"] = {
            "steps": steps, "seconds": round(secs, 2), "cell_stage_per_s": round(spec.cells * 3 * steps / secs, 1),
            "min": lo, "max": hi, "mass_change_rel_to_sum_abs": (m1 - m0) / scale, "stats": stats}
    if args.c2_fp64:
        d = np.abs(finals["fp32_mixed"] - finals["fp64"])
        out["config2_T05_fp32_vs_fp64_1024"] = {"l1": float(d.mean()), "linf": float(d.max())}
    return out


def _form_fp32(args, stream, flush, peaks):
    """Degenerate Burgers 1024^2 (the headline workload) in FP32-mixed, and the FP32-mixed
    stage on the same problem at 2048^2 and 4096^2."""
    import af_inputs as ai
    res = {}
    spec = ai.config2(1024)
    st = ai.initial_state(spec, device="cuda")
    s64, r64 = _single_form(spec, "fp64", args.form_steps, 3, st, stream, flush)
    s32, r32 = _single_form(spec, "fp32_mixed", args.form_steps, 3, st, stream, flush)
    a64, a32 = s64.device_tensors(), s32.device_tensors()
    l1 = max(float((x.double() - y.double()).abs().mean()) for x, y in zip(a32, a64))
    res["fp32_mixed_degenerate_burgers_1024"] = {
        "value": round(r32["value"], 1), "speedup_vs_fp64": round(r32["value"] / r64["value"], 2),
        "l1_vs_fp64": l1, "stage_ms_avg": round(r32["stage_ms_avg"], 5),
        "roofline": _hbm_roof("fp32_mixed", spec.cells, r32["stage_ms_avg"], peaks)}
    s64.close()
    s32.close()
    del st, a64, a32
    # the same workload on finer meshes: FP32-mixed stage throughput and HBM roofline
    for n in (2048, 4096):
        spec = ai.config2(n)
        st = ai.initial_state(spec, device="cuda", sub=2, order=3)
        s32, r32 = _single_form(spec, "fp32_mixed", args.form_steps, 3, st, stream, flush)
        res[f"fp32_mixed_degenerate_burgers_{n}"] = {
            "value": round(r32["value"], 1), "stage_ms_avg": round(r32["stage_ms_avg"], 5),
            "roofline": _hbm_roof("fp32_mixed", spec.cells, r32["stage_ms_avg"], peaks)}
        s32.close()
        del st
    return res


def _form_rk54(args, stream, flush, peaks):
    """Degenerate Burgers 1024^2 with SSP-RK(5,4), FP64 and FP32-mixed."""
    import af_inputs as ai
    spec = ai.config2(1024)
    st = ai.initial_state(spec, device="cuda")
    s64, r64 = _single_form(spec, "fp64", args.form_steps, 3, st, stream, flush, rk=54)
    s32, r32 = _single_form(spec, "fp32_mixed", args.form_steps, 3, st, stream, flush, rk=54)
    l1 = max(float((x.double() - y.double()).abs().mean()) for x, y in zip(s32.device_tensors(), s64.device_tensors()))
    res = {"rk54_degenerate_burgers_1024": {
        "fp64_value": round(r64["value"], 1), "fp32_mixed_value": round(r32["value"], 1),
        "speedup_fp32_vs_fp64": round(r32["value"] / r64["value"], 2), "l1_fp32_vs_fp64": l1,
        "roofline_fp32": _hbm_roof("fp32_mixed", spec.cells, r32["stage_ms_avg"], peaks, rk=54),
        # one limited forward-Euler evaluation's flops per stage (conservative: the fourth
        # stage's second evaluation, which shares the tau-independent work, is not counted)
        "fp64_tflops": round(FLOPS_PER_CELL_STAGE * spec.cells / (r64["stage_ms_avg"] / 1e3) / 1e12, 4)}}
    s64.close()
    s32.close()
    return res


def _form_pme(args, stream, peaks):
    """Porous medium 4096^2 from the Barenblatt profile, FP32-mixed vs FP64."""
    import af_inputs as ai
    res = {}
    spec = ai.config3(4096)
    st = ai.state_2d(lambda x, y: ai.barenblatt(x, y, 1.0), spec, device="cuda", sub=2, order=3)
    s64, r64 = _single_form(spec, "fp64", 2, 1, st, stream)
    s32, r32 = _single_form(spec, "fp32_mixed", 2, 1, st, stream)
    l1 = max(float((x.double() - y.double()).abs().mean()) for x, y in zip(s32.device_tensors(), s64.device_tensors()))
    s64.close()
    s32, r32 = _single_form(spec, "fp32_mixed", args.form_steps, 2, st, stream)
    res["fp32_mixed_pme_4096"] = {
        "value": round(r32["value"], 1), "fp64_value": round(r64["value"], 1),
        "speedup_vs_fp64": round(r32["value"] / r64["value"], 2), "l1_vs_fp64_after_3_steps": l1,
        "stage_ms_avg": round(r32["stage_ms_avg"], 5),
        "roofline": _hbm_roof("fp32_mixed", spec.cells, r32["stage_ms_avg"], peaks)}
    s32.close()
    del st
    return res


def _form_ex65():
    """Example 6.5 (1D, Dirichlet ends) as the paper runs it: 200 cells to T = 1
    through af_run, with and without double conservation (launch-bound: time to
    solution)."""
    import torch
    import af_inputs as ai
    from paper_2510_11527_gb300 import Solver
    small = {}
    for form in ("dc", "nodc"):
        spec = ai.evje_karlsen(200, diffusion_form=form)
        st = [a.numpy() for a in ai.initial_state(spec)]
        with Solver(spec, precision="fp64") as s:
            s.set_state(st)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            n = s.run(spec.T)
            torch.cuda.synchronize()
            small[form] = {"steps": n, "seconds": round(time.perf_counter() - t0, 3)}
    return {"evje_karlsen_200_to_T1": small}


def _form_examples_64_66():
    """Examples 6.4 (two hills, 100^2 to T = 4) and 6.6 (1D Buckley-Leverett, 100 cells
    to T = 1, both initial data, with and without gravity) as printed, FP64 through
    af_run: time to solution."""
    import torch
    import af_inputs as ai
    from paper_2510_11527_gb300 import Solver

    def timed(spec):
        st = [a.numpy() for a in ai.initial_state(spec)]
        with Solver(spec, precision="fp64") as s:
            s.set_state(st)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            n = s.run(spec.T)
            torch.cuda.synchronize()
            lo, _ = s.bounds()
            return {"steps": n, "seconds": round(time.perf_counter() - t0, 3), "min": lo}

    out = {"two_hills_100x100_to_T4": timed(ai.two_hills(100))}
    for g in (False, True):
        for p in ("ibvp", "rp"):
            out[f"buckley_leverett1d_{p}_{'gravity' if g else 'nogravity'}_100_to_T1"] = \
                timed(ai.buckley_leverett_1d(100, g, p))
    return out


def _form_pme3d(args, stream, peaks):
    """3D porous medium (a = u^2) from the Barenblatt profile on n3d^3 cells (default
    128^3): the four-kernel 3D stage in FP64, and the FP32-mixed form against it."""
    import statistics as st_
    import af_inputs as ai
    from paper_2510_11527_gb300 import Solver
    n = args.n3d
    spec = ai.pme_3d(n)
    host = [a.numpy() for a in ai.initial_state(spec, sub=2, order=3)]
    # the FP32-mixed form on the same workload (its L1 difference from FP64 after the
    # same timed steps)
    s32 = Solver(spec, precision="fp32_mixed")
    s32.set_stream(stream)
    s32.set_state(host)
    step32, stage32 = _time_steps(_solver_stepper(s32, stream), s32.num_stages, args.form_steps, 3, stream)
    s = Solver(spec, precision="fp64")
    s.set_stream(stream)
    s.set_state(host)
    step_ms, stage_ms = _time_steps(_solver_stepper(s, stream), s.num_stages, args.form_steps, 3, stream)
    stage_s = st_.mean(stage_ms) / 1e3
    cells = spec.cells
    out = {"cells": cells, "value": round(cells * s.num_stages * args.form_steps / (sum(step_ms) / 1e3), 1),
           "stage_ms_avg": round(st_.mean(stage_ms), 5)}
    v32 = cells * s32.num_stages * args.form_steps / (sum(step32) / 1e3)
    l1 = max(float((a.double() - b.double()).abs().mean()) for a, b in zip(s32.device_tensors(), s.device_tensors()))
    out["fp32_mixed"] = {"value": round(v32, 1), "stage_ms_avg": round(st_.mean(stage32), 5),
                         "speedup_vs_fp64": round(v32 / out["value"], 2), "l1_vs_fp64": l1}
    s32.close()
    tf = FLOPS_PER_CELL_STAGE_3D * cells / stage_s / 1e12
    gbs = BYTES_PER_CELL_STAGE_3D * cells / stage_s / 1e9
    out["roofline"] = {"bound": "alu", "achieved": round(tf, 4), "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                       "frac": round(tf / FP64_PEAK_TFLOPS, 4), "flops_per_cell_stage": FLOPS_PER_CELL_STAGE_3D,
                       "flops_note": "pure diffusion (f = 0): the count holds the diffusion, limiter and update "
                                     "operations; neither the oracle nor the CUDA stage forms the zero flux's terms",
                       "hbm_view": {"achieved_gbs": round(gbs, 1), "peak_gbs": peaks["hbm_gbs"],
                                    "frac": round(gbs / peaks["hbm_gbs"], 4),
                                    "bytes_per_cell_stage": BYTES_PER_CELL_STAGE_3D}}
    out["checks"] = {"bounds": list(s.bounds()), "stats": s.stats()}
    s.close()
    return {f"pme3d_{n}": out}


def _form_rect2d(args, stream, flush, peaks):
    """2D rectangles with outflow ends: Examples 6.7 and 6.9 as printed (100^2 to
    T = 0.5 through af_run: time to solution), and Example 6.9's problem on 2048^2 with
    outflow ends against the same mesh periodic (the cost of the ends), FP64 and
    FP32-mixed."""
    import dataclasses
    import statistics as st_
    import torch
    import af_inputs as ai
    from paper_2510_11527_gb300 import Solver
    res = {}
    small = {}
    for name, spec in (("ex67_bl", ai.buckley_leverett_2d_outflow(100)), ("ex69_blend", ai.strongly_degenerate_2d(100))):
        st = [a.numpy() for a in ai.initial_state(spec)]
        with Solver(spec, precision="fp64") as s:
            s.set_state(st)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            n = s.run(spec.T)
            torch.cuda.synchronize()
            small[name] = {"steps": n, "seconds": round(time.perf_counter() - t0, 3)}
    res["rect2d_examples_100_to_T"] = small
    n = 2048
    big = dataclasses.replace(ai.strongly_degenerate_2d(n), blend="off")
    host_rect = [a.cpu().numpy() for a in ai.initial_state(big, device="cuda", sub=2, order=3)]
    per = dataclasses.replace(big, bc="periodic")
    host_per = [host_rect[0], host_rect[1][1:, 1:].copy(), host_rect[2][:, 1:].copy(), host_rect[3][1:, :].copy()]
    out = {"cells": n * n}
    for prec in ("fp64", "fp32_mixed"):
        e = {}
        for tag, spec, st in (("outflow", big, host_rect), ("periodic", per, host_per)):
            s = Solver(spec, precision=prec)
            s.set_stream(stream)
            s.set_state(st)
            torch.cuda.synchronize()
            step_ms, stage_ms = _time_steps(_solver_stepper(s, stream), s.num_stages, args.form_steps, 3, stream, flush)
            e[tag] = {"value": round(spec.cells * s.num_stages * args.form_steps / (sum(step_ms) / 1e3), 1),
                      "stage_ms_avg": round(st_.mean(stage_ms), 5)}
            s.close()
        e["outflow_vs_periodic"] = round(e["outflow"]["value"] / e["periodic"]["value"], 3)
        out[prec] = e
    res["rect2d_strongly_degenerate_2048"] = out
    return res


def _form_bounded1d(args, stream, peaks):
    """Example 6.5's problem (1D, Dirichlet ends) on 2^24 cells: the 1D stage kernel's
    throughput, doubly conservative (FP64, FP32-mixed) and without double conservation
    (FP64)."""
    import dataclasses
    import af_inputs as ai
    res = {}
    n = args.n1d
    big = ai.evje_karlsen(n)
    sd = ai.state_1d(ai.evje_karlsen_fn, big, device="cuda", sub=2, order=3)
    out = {"cells": n}
    r = {}
    for prec, form in (("fp64", "dc"), ("fp64", "nodc"), ("fp32_mixed", "dc")):
        spec = dataclasses.replace(big, diffusion_form=form)
        s, rr = _single_form(spec, prec, args.form_steps, 3, sd, stream)
        r[(prec, form)] = (s, rr)
        stage_s = rr["stage_ms_avg"] / 1e3
        e = {"value": round(rr["value"], 1), "stage_ms_avg": round(rr["stage_ms_avg"], 5),
             "hbm_gbs": round(BYTES_PER_CELL_STAGE_1D[prec] * n / stage_s / 1e9, 1),
             "hbm_frac": round(BYTES_PER_CELL_STAGE_1D[prec] * n / stage_s / 1e9 / peaks["hbm_gbs"], 4)}
        if prec == "fp64":
            tf = FLOPS_PER_CELL_STAGE_1D[form] * n / stage_s / 1e12
            e["roofline"] = {"bound": "alu", "achieved": round(tf, 4), "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                             "frac": round(tf / FP64_PEAK_TFLOPS, 4),
                             "flops_per_cell_stage": FLOPS_PER_CELL_STAGE_1D[form]}
        out[f"{prec}_{form}"] = e
    a64 = r[("fp64", "dc")][0].device_tensors()
    a32 = r[("fp32_mixed", "dc")][0].device_tensors()
    out["fp32_mixed_dc"]["l1_vs_fp64"] = max(float((x.double() - y.double()).abs().mean()) for x, y in zip(a32, a64))
    out["fp32_mixed_dc"]["speedup_vs_fp64"] = round(out["fp32_mixed_dc"]["value"] / out["fp64_dc"]["value"], 2)
    for s, _ in r.values():
        s.close()
    del sd, a64, a32
    res[f"bounded1d_evje_karlsen_{n}"] = out
    return res


def _batch_run(inst, prec, steps, blend=0):
    """Build the batch in precision `prec` (blend 0 off, 1 plain, 2 learned: a seeded
    network of random weights -- the cost does not depend on them), autotune its tile,
    time `steps` graph-replayed steps; returns (cell-stage/s, cells, tile, ms per step,
    safeguard errors)."""
    import torch
    import af_inputs as ai
    from paper_2510_11527_gb300 import capi
    grids, fl, df, bd = [], [], [], []
    for s_, _ in inst:
        grids.append(capi.af_grid(2, s_.nx, s_.ny, s_.x0, s_.x1, s_.y0, s_.y1))
        f = capi.af_flux()
        f.kind = capi.FLUX[s_.flux[0]]
        f.p[0] = s_.flux[1][0]
        d = capi.af_diff()
        d.kind = capi.DIFF[s_.diff[0]]
        for k, v in enumerate(s_.diff[1]):
            d.p[k] = v
        fl.append(f)
        df.append(d)
        bd.append(capi.af_bounds_t(s_.umin, s_.umax, 0))
    opts = capi.af_opts(capi.PREC[prec], 3, 0.0, 0.0, 1, blend, 1.0)
    b = capi.af_batch_create(grids, fl, df, bd, opts)
    net = None
    try:
        if blend == 2:
            net = capi.af_mlp_create()
            capi.af_mlp_set_params(net, ai.mlp_init_params(6))
            capi.af_batch_set_mlp(b, net)
        cells = 0
        for i, (s_, modes) in enumerate(inst):
            stt = ai.batch_state(s_, modes, device="cuda")
            ptrs, (_, pb) = capi.af_batch_device_ptrs(b, i)
            shp = (s_.ny, s_.nx)
            for k, (p, src) in enumerate(zip(ptrs, stt)):
                _cuda_view(p, shp, "<f8" if (k == 0 or pb == 8) else "<f4").copy_(src)
            cells += s_.cells
        torch.cuda.synchronize()
        tile = capi.af_batch_autotune(b)
        capi.af_batch_step(b, 2)
        capi.af_batch_sync(b)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        # the batch runs on its own stream; record around a synchronised replay
        e0.record()
        capi.af_batch_step(b, steps)
        capi.af_batch_sync(b)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        return cells * 3 * steps / (ms / 1e3), cells, tile, ms / steps, capi.af_batch_stats(b)["errors"]
    finally:
        capi.af_batch_destroy(b)
        if net is not None:
            capi.af_mlp_destroy(net)


def _form_batch(args, stream, headline_value, peaks):
    """256 uneven instances (FP32-mixed and FP64), graph replay, autotuned tile; the
    FP32-mixed batch also with the plain and the learned blend."""
    import af_inputs as ai
    inst = ai.batch_instances()
    val, cells, tile, ms_step, errors = _batch_run(inst, "fp32_mixed", args.form_steps)
    v64, _, tile64, _, err64 = _batch_run(inst, "fp64", max(1, args.form_steps // 2))
    vp, _, tp, _, errp = _batch_run(inst, "fp32_mixed", args.form_steps, blend=1)
    vl, _, tl, _, errl = _batch_run(inst, "fp32_mixed", args.form_steps, blend=2)
    return {"batch_256_fp32_mixed": {
        "value": round(val, 1), "cells": cells, "tile": list(tile), "ms_per_step": round(ms_step, 4),
        "fp64_value": round(v64, 1), "fp64_tile": list(tile64), "speedup_vs_fp64": round(val / v64, 2),
        "speedup_vs_fp64_single_mesh": round(val / headline_value, 2),
        "plain_blend_value": round(vp, 1), "plain_blend_tile": list(tp),
        "learned_blend_value": round(vl, 1), "learned_blend_tile": list(tl),
        "safeguard_errors": errors + err64 + errp + errl,
        "roofline": _hbm_roof("fp32_mixed", cells, ms_step / 3, peaks)}}


def _form_bl(args, stream, peaks):
    """Buckley-Leverett 4096^2: plain vs learned blend (trained here), FP32-mixed."""
    import torch
    import af_inputs as ai
    from paper_2510_11527_gb300 import capi
    res = {}
    net = capi.af_mlp_create()
    try:
        capi.af_mlp_set_params(net, ai.mlp_init_params(1))
        feats, labels = [], []
        # 64 random piecewise-constant fields of 128^2 cells: 1.05e6 method-labelled patches
        for k in range(64):
            sp = ai.config5(128)
            sp.blend = "plain"
            stt = ai.random_piecewise(sp, seed=100 + k, device="cuda")
            s_, _ = _single_form(sp, "fp32_mixed", 4, 0, stt, stream)
            f = torch.empty((sp.cells, 21), dtype=torch.float32, device="cuda")
            lab = torch.empty(sp.cells, dtype=torch.float32, device="cuda")
            capi.af_mlp_features(s_.ctx, f.data_ptr(), lab.data_ptr())
            feats.append(f)
            labels.append(lab)
            s_.close()
        X, Y = torch.cat(feats), torch.cat(labels)
        t0 = time.perf_counter()
        loss = capi.af_mlp_train(net, X.data_ptr(), Y.data_ptr(), X.shape[0], 4096, 1500, 3e-3, 8)
        train_s = time.perf_counter() - t0
        spec = ai.config5(4096)
        st = ai.state_2d(ai.bl_disc_fn, spec, device="cuda", sub=2, order=3)
        spec.blend = "plain"
        sp_, rp = _single_form(spec, "fp32_mixed", args.form_steps, 2, st, stream)
        spec_l = ai.config5(4096)
        spec_l.blend = "external"
        sl_, rl = _single_form(spec_l, "fp32_mixed", args.form_steps, 2, st, stream, net=net)
        l1 = float((sl_.device_tensors()[0] - sp_.device_tensors()[0]).abs().mean())
        sp_.close()
        sl_.close()
        spec.blend = "plain"
        s64, r64 = _single_form(spec, "fp64", 2, 1, st, stream)
        s64.close()
        res["bl_4096_fp32_mixed"] = {
            "plain_blend_value": round(rp["value"], 1), "learned_blend_value": round(rl["value"], 1),
            "fp64_plain_value": round(r64["value"], 1),
            "speedup_plain_vs_fp64": round(rp["value"] / r64["value"], 2),
            "speedup_learned_vs_fp64": round(rl["value"] / r64["value"], 2),
            "l1_learned_vs_plain": l1, "train": {"samples": int(X.shape[0]), "steps": 1500, "final_loss": loss,
                                                   "seconds": round(train_s, 2)},
            "roofline_plain": _hbm_roof("fp32_mixed", spec.cells, rp["stage_ms_avg"], peaks),
            "roofline_learned": _hbm_roof("fp32_mixed", spec.cells, rl["stage_ms_avg"], peaks)}
    finally:
        capi.af_mlp_destroy(net)
    return res


def _oracle_proc(bar, q, steps, seconds, warmup):
    """One host core: the FP64 oracle, as it stands (single-threaded), on its own copy of
    the bounded sample (degenerate Burgers at 512^2), timed after all workers are ready."""
    import af_inputs as ai
    import oracle
    spec = ai.config2(512)
    st = [a.numpy() for a in ai.initial_state(spec)]
    dt = oracle.dt_cfl(spec, st[0])
    for _ in range(max(1, warmup)):
        st, _ = oracle.step(spec, 3, st, dt)
    bar.wait()
    t0 = time.perf_counter()
    n = 0
    while (n < steps) if steps else (time.perf_counter() - t0 < seconds):
        st, _ = oracle.step(spec, 3, st, dt)
        n += 1
    q.put((spec.cells * 3 * n, n, time.perf_counter() - t0))


def oracle_on_host_cores(steps=None, seconds=None, workers=None, warmup=1):
    """Run one oracle process per host core (spawned, so no forked CUDA state) and return
    (cell-stages/s over all cores, per-core mean, cores, steps per core, wall seconds)."""
    import multiprocessing as mp
    n = workers or len(os.sched_getaffinity(0))
    ctx = mp.get_context("spawn")
    bar, q = ctx.Barrier(n), ctx.Queue()
    procs = [ctx.Process(target=_oracle_proc, args=(bar, q, steps, seconds, warmup)) for _ in range(n)]
    for p in procs:
        p.start()
    res = [q.get() for _ in range(n)]
    for p in procs:
        p.join()
    wall = max(r[2] for r in res)
    total = sum(r[0] for r in res) / wall
    per_core = statistics.mean(r[0] / r[2] for r in res)
    return total, per_core, n, min(r[1] for r in res), wall


def cpu_sample(seconds_target=12.0):
    """The FP64 oracle on every host core, each core on a bounded sample of the workload
    (config 2 at 512^2) for about seconds_target."""
    total, per_core, n, steps, wall = oracle_on_host_cores(seconds=seconds_target)
    return {"value": round(total, 1), "unit": UNIT, "cores": n, "kind": "oracle", "per_core_value": round(per_core, 1),
            "sample": f"degenerate_burgers2d 512x512 FP64 SSP-RK3, one single-threaded oracle process per core, "
                      f">= {steps} steps each ({wall:.1f} s)"}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return None
    total, per_core, n, steps, wall = oracle_on_host_cores(steps=args.steps, warmup=args.warmup)
    # one "step" = one SSP-RK3 step of the 512^2 sample on every host core
    import af_inputs as ai
    cells = ai.config2(512).cells
    return {"impl": "reference", "metric": METRIC, "value": round(total, 1), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(wall / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "degenerate_burgers2d_512x512_fp64_ssprk3_mpp on every host core "
                                   "(bounded sample of the 1024^2 workload)", "cells_per_core": cells},
            "cpu_baseline": {"value": round(total, 1), "unit": UNIT, "cores": n, "kind": "oracle",
                             "per_core_value": round(per_core, 1),
                             "sample": f"512x512 cells per core, {args.steps} SSP-RK3 steps, one process per core"},
            "e2e": {"value": round(total, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32_mixed"])
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--workload", default="degenerate_burgers",
                    choices=["degenerate_burgers", "buckley_leverett_plain_blend"],
                    help="the timed workload: config 2 (default) or Buckley-Leverett with the plain blend")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the FP32/batched/learned forms")
    ap.add_argument("--form-steps", type=int, default=5)
    ap.add_argument("--n1d", type=int, default=1 << 24, help="cells of the bounded1d form")
    ap.add_argument("--n3d", type=int, default=128, help="cells per direction of the pme3d form")
    ap.add_argument("--pme-n", type=int, default=2048, help="FP32-mixed mesh of the pme_full form (run to t = 2)")
    ap.add_argument("--c2-fp64", action="store_true", help="c2_full form: also run FP64 to T = 0.5 (about 4 min)")
    ap.add_argument("--forms", default="fp32,rk54,pme,batch,bl,bounded1d,ex65,ex64_66,rect2d,pme3d",
                    help="comma list of forms to run: fp32 (Burgers 1024^2), rk54 (Burgers 1024^2 with "
                         "SSP-RK(5,4)), pme (4096^2), batch (256), bl (4096^2), bounded1d (Example 6.5's "
                         "problem on 2^24 cells, with and without double conservation), ex65 (Example 6.5 "
                         "as printed: 200 cells to T = 1), ex64_66 (Examples 6.4 and 6.6 as printed), rect2d (Examples 6.7 / 6.9 at 100^2 to T and "
                         "Example 6.9's problem on 2048^2 with outflow ends vs periodic), pme3d (3D porous "
                         "medium on 128^3)")
    args = ap.parse_args()
    if args.impl == "reference":
        res = run_reference(args)
        if res is not None:
            print(json.dumps(res))
        return
    res = run_gpu(args)
    if res is not None:
        rank, world, _ = dist_env()
        if not args.no_forms and world == 1:
            peaks, _ = load_peaks()
            res["forms"] = forms(args, res["value"], peaks)
        if not args.no_cpu_baseline and world == 1:
            res["cpu_baseline"] = cpu_sample()
        print(json.dumps(res))


if __name__ == "__main__":
    main()
