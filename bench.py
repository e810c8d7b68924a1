"""Benchmark: RIDC-4 on 2048x2048 Gray-Scott, mixed BF16x3 solves, cell-updates per second.

One bench step is one whole integration: every level is reset to the initial field and the
pipeline advances until the most corrected level has taken 1000 steps of dt = 0.5 (start-up
and drain included), i.e. 2048^2 * 1000 cell-updates. `value` times that on the device with
inputs resident in HBM; `e2e` times the same through the C ABI with host buffers (initial
field copied in, solution copied out inside the timed region).

Also reported: the dominant kernel's roofline (CUDA events around every launch inside the
timed region), the FP64 GPU form of the same workload on a truncated run together with the
mixed path's relative L2 difference to it, SM clocks sampled during the timed region, and the
CPU oracle on a bounded sample of the workload (reference arm: --impl reference).

Multi-GPU (torchrun): the integration does not shard; every rank runs an independent replica
and `value` sums the ranks' cell-updates over the slowest rank's time (weak scaling).
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RIDC-4 cell-updates/s, 2048² Gray-Scott: mixed vs FP64 GPU at <=1e-8 rel L2"
UNIT = "cell-updates/s"
N, NT, ORDER, NREF = 2048, 1000, 4, 2
PROF_EVERY = 8
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def _peaks():
    try:
        with open(PEAKS_FILE) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def whole_job_rate(local_ms: float, units_per_rank: float, device=None) -> tuple[float, float]:
    """(units/s over all ranks, slowest rank's ms): every rank processed `units_per_rank`
    units in `local_ms`; the job's rate is the units of all ranks over the slowest rank's
    time (replicas, weak scaling). Works with any torch.distributed backend (gloo on CPU
    tensors, NCCL on CUDA tensors), or without a process group."""
    import torch
    import torch.distributed as dist
    ws = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    slow = float(t.item())
    return ws * units_per_rank / (slow * 1e-3), slow


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while active."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix="ridc_clocks_", suffix=".csv")
        os.close(fd)

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={CLOCK_QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), float(f[3]), f[4:]))
            except ValueError:
                continue
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [r for r in rows if r[2] > 200.0] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in loaded for i, v in enumerate(r[3][1:5])
                          if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in loaded),
                "sm_max_mhz": max(r[1] for r in rows), "samples": len(loaded),
                "power_w_max": max(r[2] for r in rows), "reasons": reasons}


# DRAM traffic of one full (8-plane) gemm_sym launch from one ncu capture
# (profiles/gemm_sym_gray_scott_2048_mixed.md: dram__bytes_read.sum + dram__bytes_write.sum,
# mean over the four modes), valid only for the kernel source it was taken on.
GEMM_TRAFFIC = {"bytes": 2.3186e8,
                "source_sha256": "04f824db85932070ed0507afae62ae4893e1183ec26bed1aa57c393238153959"}


def gemm_traffic():
    """Per-launch DRAM bytes of gemm_sym, or None once its source differs from the one the
    counters were taken on."""
    import hashlib
    path = os.path.join(ROOT, "paper_1209_4297_gb300", "csrc", "gemm_sym.cu")
    try:
        digest = hashlib.sha256(open(path, "rb").read()).hexdigest()
    except OSError:
        return None
    return GEMM_TRAFFIC["bytes"] if digest == GEMM_TRAFFIC["source_sha256"] else None


# FP64 pipe of GB300: 2 FP64 operations (DADD, DMUL or DFMA) per clock per SM, i.e. the
# nominal 1.25 TFLOP/s (FMA = 2 flop) at 152 SMs x 2070 MHz.
FP64_OPS_PER_CLK_SM = 2


def step_work(masks, species=2, order=ORDER, nref=NREF, n=N):
    """Algorithmic FP64 operations and bytes of the non-GEMM kernels of the mixed
    Gray-Scott path, summed over the pipeline steps in `masks` (bit j: level j advances).
    Per plane-cell (one species of one advancing level):
      rhs       predictor 1 op (dt F), corrector j: 2 differences, dt fma, j+1 quadrature
                fmas = j+4 ops; reads 1 (predictor) or j+5 FP64 fields, writes r (8 B) and
                the split operand (4 B)
      residual  first pass 5 ops (stencil: 3 adds, 2 fmas), later passes 6 (+1 add for
                delta = previous + increment); reads r (8 B), increment (4 B) and from the
                second pass the previous delta (8 B), writes delta (8 B) and the split (4 B)
      finalize  eta = base + d64 + d32 (2 adds), f = f^N + D eta on levels that keep f
                (3 adds, 2 fmas), plus the reaction per cell (u v^2: 2 muls; 1 add, 2 fmas);
                reads base, d64, d32 (20 B), writes eta, f^N and f where kept (8 B each)."""
    cells = float(n * n)
    ops = {"rhs": 0.0, "residual": 0.0, "finalize": 0.0}
    byt = dict(ops)
    for m in masks:
        act = [j for j in range(order) if (int(m) >> j) & 1]
        for j in act:
            keeps_f = j < order - 1 or j == 0
            ops["rhs"] += (1 if j == 0 else j + 4) * species * cells
            byt["rhs"] += ((8 if j == 0 else 8 * (j + 5)) + 12) * species * cells
            ops["residual"] += (5 + 6 * (nref - 1)) * species * cells
            byt["residual"] += (24 + 32 * (nref - 1)) * species * cells
            ops["finalize"] += (2 * species + 5 + (5 * species if keeps_f else 0)) * cells
            byt["finalize"] += (20 + 16 + (8 if keeps_f else 0)) * species * cells
    return ops, byt


def fp64_kernel_rooflines(masks, stats, runs, peaks):
    """Achieved FP64-pipe and HBM rates of the non-GEMM kernels over the timed region."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak_ops = FP64_OPS_PER_CLK_SM * sms * mhz * 1e6
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    ops, byt = step_work(masks)
    out = {"bound": "alu", "unit": "FP64 op/s (DADD, DMUL, DFMA each 1)", "peak": peak_ops,
           "peak_source": f"{FP64_OPS_PER_CLK_SM} FP64 ops/clk/SM x {sms} SMs x {mhz:.0f} MHz "
                          "(nominal 1.25 TFLOP/s)", "kernels": {}}
    for k in ops:
        launches, ms = stats[k]
        if ms <= 0:
            continue
        s = ms * 1e-3
        ent = {"launches": launches, "ms": ms,
               "hbm_gbs": runs * byt[k] / s / 1e9, "hbm_frac": runs * byt[k] / s / 1e9 / hbm}
        if ops[k] > 0:
            ent["fp64_ops_per_s"] = runs * ops[k] / s
            ent["fp64_frac"] = runs * ops[k] / s / peak_ops
        out["kernels"][k] = ent
    return out


def cpu_baseline(steps: int = 6, threads: int = 1):
    """The FP64 oracle (sequential classic-IDC order, numpy/scipy) on 2048^2 Gray-Scott.
    threads > 1 lets scipy.fft's transforms (the oracle's solves) use that many threads;
    the oracle's numpy arithmetic stays single-threaded either way."""
    import scipy.fft

    import inputs
    import oracle
    w = inputs.gray_scott_2d(n=N, nsteps=steps)
    prob = oracle.from_workload(w)
    with scipy.fft.set_workers(threads):
        t0 = time.perf_counter()
        oracle.ridc_sequential(prob, w.u0, w.dt, steps, ORDER)
        dt = time.perf_counter() - t0
    how = "single thread" if threads == 1 else f"scipy.fft on {threads} threads"
    return {"value": N * N * steps / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{steps} RIDC-4 steps of the 2048^2 Gray-Scott workload "
                      f"({dt:.1f} s, numpy/scipy FP64, {how})"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    vals = []
    for _ in range(args.warmup):
        cpu_baseline(args.ref_steps)
    for _ in range(args.steps):
        vals.append(cpu_baseline(args.ref_steps))
    v = statistics.median(x["value"] for x in vals)
    cb = dict(vals[0])
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * N * N * args.ref_steps / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "gray_scott_2048_ridc4_mixed", "grid": N, "species": 2,
                       "order": ORDER, "top_level_steps": NT, "dt": 0.5, "n_refine": NREF,
                       "parallelism": "replicas x1",
                       "reference_sample": f"{args.ref_steps} top-level steps of the workload "
                                           "per timed step: the FP64 CPU oracle (sequential "
                                           "IDC order, exact FP64 solves)"},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ensemble(args):
    """The 512-instance ensemble (uneven Dirichlet advection-diffusion, solves at FP32 accuracy
    on the tensor cores (TF32 hi/lo, three products) with two FP64-residual refinement passes:
    with one, the worst instance misses the 1e-8 bar) advanced 256 steps by one persistent
    launch; the autotuner
    picks the launch configuration first. Not the default line: a per-config measurement.
    --ens-count / --ens-steps shrink it (for profiling a small case)."""
    import torch

    import inputs
    from paper_1209_4297_gb300 import Batch

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    count, nst = args.ens_count, args.ens_steps
    ws = inputs.ensemble(count, nsteps=nst)
    u0s = [torch.from_numpy(w.u0[0].copy()).cuda() for w in ws]
    b = Batch(ws, n_refine=args.ens_refine, stream=stream.cuda_stream)
    b.set_initial(u0s)
    choice, tune_ms = b.autotune(8)
    tiles = {str(side): b.tile_width(side) for side in sorted({w.n for w in ws})}
    cells = b.cells()
    for _ in range(args.warmup):
        b.set_initial(u0s)
        b.advance(nst)
    torch.cuda.synchronize()
    times = []
    g0 = b.graph_launches()
    with ClockSampler(0) as clk:
        for _ in range(args.steps):
            b.set_initial(u0s)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.advance(nst)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
    graphs = b.graph_launches() - g0
    ms = statistics.median(times)
    # the oracle on a bounded sample: four instances (smallest work, a middle one, the
    # largest, and the one with the strongest growth) over the first k steps; its time is
    # the CPU baseline and its results the reference of the relative L2
    import oracle
    k_or = min(nst, args.oracle_steps or 16)
    b.set_initial(u0s)
    b.advance(k_or)
    work = [w.order * w.n ** 3 for w in ws]
    picks = sorted({int(np.argmin(work)), int(np.argsort(work)[len(ws) // 2]),
                    int(np.argmax(work)), min(303, len(ws) - 1)})
    rels, s_or, cells_or = [], 0.0, 0
    for i in picks:
        w = ws[i]
        t0 = time.perf_counter()
        ref = oracle.ridc_sequential(oracle.from_workload(w), w.u0, w.dt, k_or, w.order)[0]
        s_or += time.perf_counter() - t0
        cells_or += w.n * w.n * k_or
        got = b.solution(i)
        rels.append(float(np.linalg.norm(got - ref) / np.linalg.norm(ref)))
    b.close()
    cpu = {"value": cells_or / s_or, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"instances {picks}, {k_or} steps each ({s_or:.1f} s, numpy/scipy FP64, "
                     "single thread)"}
    # algorithmic work of the launch. Solves: per advancing level and pass, four transforms,
    # each two parity-split (side x side/2) x (side/2 x side/2) products = side^3 flop, run as
    # three TF32 split products. FP64 phases, per cell of an advancing level (ens_step_ops):
    # right-hand side 1 (predictor) or j+4, per refinement pass the residual stencil (5) and
    # the running total (1 from the second pass), new state 2, f^N 4 and f 5 (levels that
    # keep f).
    from paper_1209_4297_gb300 import schedule_plan
    passes = 1 + args.ens_refine
    gemm_flops, fp64_ops = 0.0, 0.0
    for w in ws:
        for m in schedule_plan(w.order, nst):
            for j in range(w.order):
                if not (int(m) >> j) & 1:
                    continue
                gemm_flops += 4 * 1.0 * w.n ** 3 * passes
                keeps_f = j < w.order - 1 or j == 0
                ops = ((1 if j == 0 else j + 4) + 5 * args.ens_refine + max(0, args.ens_refine - 1)
                       + 2 + 4 + (5 if keeps_f else 0))
                fp64_ops += ops * w.n * w.n
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    peaks, peak_src = _peaks()
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    fp64_peak = FP64_OPS_PER_CLK_SM * sms * mhz * 1e6
    tf32_peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops")) / 2   # TF32 = BF16 / 2
    secs = ms * 1e-3
    gemm_tf = gemm_flops / secs / 1e12
    line = {"metric": f"ensemble cell-updates/s (sum over instances of side^2 x {nst} steps)",
            "value": cells * nst / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "dtype": "f64+tf32x3(fp32 acc) solves", "data": "synthetic", "gpu_launches": int(graphs),
            "gpu_launches_note": "CUDA graphs of one persistent cluster kernel each",
            "scaling": "weak", "vs_baseline": None,
            "rel_l2_vs_oracle": {"value": max(rels), "instances": picks,
                                 "per_instance": rels, "top_level_steps": k_or},
            "cpu_baseline": None if args.no_cpu else cpu, "clocks": clk.summary(),
            "config": {"workload": f"ensemble_{count}_dirichlet_adv_diff", "instances": count,
                       "steps": nst, "n_refine": args.ens_refine, "autotune_choice": choice,
                       "tile_widths": tiles,
                       "launch": "one CUDA graph per advance (counter reset + persistent "
                                 "cluster launch)",
                       "cells_per_step": cells},
            "roofline": {"bound": "alu", "kernel": "ensemble_kernel (one persistent cluster "
                         "launch: FP64 phases and TF32x3 tcgen05 solves)",
                         "achieved": fp64_ops / secs, "peak": fp64_peak, "unit": "FP64 op/s",
                         "frac": fp64_ops / secs / fp64_peak,
                         "peak_source": f"{FP64_OPS_PER_CLK_SM} FP64 ops/clk/SM x {sms} SMs x "
                                        f"{mhz:.0f} MHz (nominal FP64 pipe)",
                         "work": "FP64 operations per cell of an advancing level: right-hand "
                                 "side 1 or j+4, 5 per refinement residual (+1 running total "
                                 "from the second pass), new state 2, f^N 4, f 5",
                         "tensor": {"achieved_useful_tflops": gemm_tf,
                                    "issued_tflops": 3 * gemm_tf, "peak": tf32_peak,
                                    "frac_issued": 3 * gemm_tf / tf32_peak,
                                    "peak_source": f"{peak_src} bf16_tflops_sustained / 2 "
                                                   "(dense TF32 is half of BF16)"},
                         "traffic": None,
                         "note": "the whole launch, FP64 phases and solves together; neither "
                                 "pipe is saturated: per-instance phases are separated by "
                                 "cluster barriers"}}
    print(json.dumps(line), flush=True)


# ---- per-config lines -----------------------------------------------------------------------
# Algorithmic FP64 operations per cell of one level-step of the 1D kernel (an approximate count
# of the operations the algorithm needs, stated so the FP64-pipe fraction can be checked):
# right-hand side 1 (predictor, dt F) or j+4 (corrector j: two differences, one dt fma, j+1
# quadrature fmas); solve 8 (backward recurrence and its carry, cyclic wrap, forward recurrence
# with its rho/mu scaling, carry and wrap); new state 1; f^N 2 and F 4.
ONED_SOLVE_OPS, ONED_STATE_OPS = 8, 7


def planes_solved(mask: int, order: int, species: int, stages: int) -> int:
    """Plane-solves of one pipeline step: every advancing level solves its species once, an
    ARK predictor's level solves once per implicit stage (stages - 1)."""
    act = [j for j in range(order) if (mask >> j) & 1]
    n = 0
    for j in act:
        n += species * ((stages - 1) if (j == 0 and stages > 1) else 1)
    return n


def oned_ops(masks, order, n):
    """Algorithmic FP64 operations of a 1D integration (counts above)."""
    ops = 0.0
    for m in masks:
        for j in range(order):
            if (int(m) >> j) & 1:
                ops += ((1 if j == 0 else j + 4) + ONED_SOLVE_OPS + ONED_STATE_OPS) * n
    return ops


def _timed_integrations(it, u0, nt, runs, stream, prof):
    """CUDA-event time (ms) of `runs` whole integrations from u0 (inputs resident), with
    nvidia-smi clocks sampled meanwhile and kernel timing at period `prof`."""
    import torch
    it.set_profiling(prof)
    launches0 = it.launch_count()
    times = []
    with ClockSampler(torch.cuda.current_device()) as clk:
        for _ in range(runs):
            it.set_initial(u0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            it.advance(nt)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
    kinds = ("rhs", "gemm_tc", "gemm_f64", "residual", "finalize", "ridc1d", "split_f16")
    stats = {k: it.kernel_stats(k) for k in kinds}
    it.set_profiling(False)
    return times, it.launch_count() - launches0, stats, clk.summary()


def run_single(args):
    """One of the other single-instance workloads, timed like the default line (whole
    integrations, CUDA events, inputs resident, clocks sampled), with its dominant kernel's
    roofline, the oracle on a bounded sample of the same workload (its time is the CPU
    baseline, its result the reference of the line's relative L2), and for the 1D workloads
    the same pipeline with one level (FBE) for the paper's wall-time comparison:
      adv_diff_1d          the 1D periodic workload (N = 256, 512 steps, FP64)
      adv_diff_upwind_1d   the paper's upwind advection-diffusion run (T = 40, 10 restarts)
      burgers_1d           the paper's viscous Burgers run (T = 1)
      gray_scott_1024_fp64 1024^2 Gray-Scott in FP64, all 2000 steps
      gray_scott_2048_mixed the headline grid in a chosen form (--mixed-precision, --n-refine,
                           --order, --predictor)
      adv_diff_4096        the 4096^2 Dirichlet workload (512 steps, mixed)
    --predictor ark3 / ark4 runs any of them with an ARK predictor (Theorem 2)."""
    import torch

    import inputs
    import oracle
    from paper_1209_4297_gb300 import Integrator, schedule_plan_predictor

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    if args.workload == "adv_diff_1d":
        w, prec, nt = inputs.adv_diff_1d(), "fp64", 512
    elif args.workload == "adv_diff_upwind_1d":
        w, prec, nt = inputs.adv_diff_upwind_1d(), "fp64", 4000
    elif args.workload == "burgers_1d":
        w, prec, nt = inputs.burgers_1d(), "fp64", 2000
    elif args.workload == "gray_scott_1024_fp64":
        w, prec, nt = inputs.gray_scott_2d(n=1024, nsteps=2000), "fp64", 2000
    elif args.workload == "gray_scott_2048_mixed":
        w, prec, nt = inputs.gray_scott_2d(n=2048, nsteps=1000), args.mixed_precision, args.nt
    else:
        w, prec, nt = inputs.adv_diff_2d(n=4096, nsteps=512), args.mixed_precision, 512
    order = args.order or w.order
    pred = args.predictor
    stages = {"fbe": 1, "ark3": 5, "ark4": 7}[pred]
    S = w.species
    u0 = torch.from_numpy(w.u0).cuda()
    kw = dict(precision=prec, n_refine=args.n_refine, stream=stream.cuda_stream)

    # warm-up: W integrations, at most 40 steps each for the long lines (tables, caches and
    # clocks are warm after the first); then K whole integrations are timed
    warm_nt = nt if nt <= 600 else 40
    it = Integrator.from_workload(w, order=order, predictor=pred, **kw)
    for _ in range(args.warmup):
        it.set_initial(u0)
        it.advance(warm_nt)
    torch.cuda.synchronize()
    prof = 1 if w.dim == 1 else PROF_EVERY
    times, launches, stats, clocks = _timed_integrations(it, u0, nt, args.steps, stream, prof)
    ms = statistics.median(times)
    cells_side = w.n if w.dim == 1 else w.n * w.n
    cells = cells_side * nt
    masks = schedule_plan_predictor(order, pred, nt)
    peaks, peak_src = _peaks()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    fp64_peak = FP64_OPS_PER_CLK_SM * sms * mhz * 1e6

    # ---- roofline of the dominant kernel (work of the sampled steps over their launch time)
    sampled = masks[::prof]
    passes = 1 if prec == "fp64" else 1 + args.n_refine
    roof = None
    if w.dim == 1:
        n_l, ms_l = stats["ridc1d"]
        cl = min(order, 8)
        ops = oned_ops(masks, order, w.n) * args.steps
        peak = FP64_OPS_PER_CLK_SM * cl * mhz * 1e6
        if ms_l > 0:
            roof = {"bound": "alu", "kernel": "ridc1d_kernel (one SM per level, cluster of "
                    f"{cl})", "achieved": ops / (ms_l * 1e-3), "peak": peak,
                    "unit": "FP64 op/s", "frac": ops / (ms_l * 1e-3) / peak,
                    "peak_source": f"{FP64_OPS_PER_CLK_SM} FP64 ops/clk/SM x {cl} SMs x "
                                   f"{mhz:.0f} MHz (the SMs the launch uses)",
                    "work": "about (rhs + 8 solve + 7 state) FP64 ops per cell per level-step",
                    "traffic": None,
                    "note": "latency-bound: a step is a chain of block-wide scans and one "
                            "cluster barrier"}
    elif prec == "fp64":
        n_g, ms_g = stats["gemm_f64"]
        per = 4.0 * w.n ** 3 if w.n % 2 == 0 else 8.0 * w.n ** 3   # per plane-solve
        flops = sum(planes_solved(int(m), order, S, stages) for m in sampled) * per * args.steps
        if ms_g > 0:
            ach = flops / (ms_g * 1e-3)
            roof = {"bound": "alu", "kernel": "gemm_f64_split_kernel (parity-split DFMA fast "
                    "diagonalisation)", "achieved": ach / 1e12, "peak": 2 * fp64_peak / 1e12,
                    "unit": "TFLOP/s", "frac": ach / (2 * fp64_peak),
                    "peak_source": f"{FP64_OPS_PER_CLK_SM} DFMA/clk/SM x {sms} SMs x "
                                   f"{mhz:.0f} MHz x 2 flop (nominal FP64 pipe)",
                    "work": "N^3 flop per plane per transform (parity split), 4 transforms "
                            "per solve", "traffic": None,
                    "avg_launch_ms": ms_g / n_g if n_g else None}
    else:
        n_t, ms_t = stats["gemm_tc"]
        flops = (sum(planes_solved(int(m), order, S, stages) for m in sampled)
                 * 4 * passes * 3.0 * w.n ** 3 * args.steps)
        peak_tf = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
        if ms_t > 0:
            ach = flops / (ms_t * 1e-3) / 1e12
            roof = {"bound": "tensor", "kernel": "gemm_sym_kernel (parity-split "
                    f"{prec[6:].upper()} tcgen05)", "achieved": ach, "peak": peak_tf,
                    "unit": "TFLOP/s", "frac": ach / peak_tf,
                    "peak_source": f"{peak_src} bf16_tflops_sustained",
                    "useful_tflops": ach / 3, "work": "3 N^3 flop per plane per transform "
                    "(three split products), 4 transforms per pass", "traffic": None,
                    "avg_launch_ms": ms_t / n_t if n_t else None}
    share = {k: {"launches": v[0], "ms": v[1]} for k, v in stats.items() if v[0]}

    # ---- FBE on the same path (1D: the paper's wall-time comparison)
    fbe_ms = None
    if w.dim == 1 and order > 1:
        it1 = Integrator.from_workload(w, order=1, **kw)
        t1, _, _, _ = _timed_integrations(it1, u0, nt, args.steps, stream, 0)
        it1.close()
        fbe_ms = statistics.median(t1)

    # ---- the oracle on a bounded sample: CPU baseline and the reference of the rel. L2
    if w.dim == 1:
        k_or = nt                                  # the whole workload
    elif w.n <= 1024:
        k_or = args.oracle_steps or 12
    else:
        k_or = args.oracle_steps or 2
    it.set_initial(u0)
    it.advance(k_or)
    got = it.solution()
    it.close()
    t0 = time.perf_counter()
    ref = oracle.ridc_restarted(oracle.from_workload(w), w.u0, w.dt, k_or, order,
                                w.restart_every, predictor=pred)
    s_or = time.perf_counter() - t0
    # the oracle runs its lower levels ahead to the top level's start-up nodes, so its rate
    # counts the top level's steps only, as the GPU line does
    cpu = {"value": cells_side * k_or / s_or, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{k_or} top-level steps of this workload ({s_or:.1f} s, numpy/scipy "
                     "FP64, single thread)"}
    rel = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))

    line = {"metric": f"RIDC-{order} cell-updates/s" + ("" if pred == "fbe" else
                                                         f", {pred.upper()} predictor"),
            "value": cells / (ms * 1e-3), "unit": UNIT,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "us_per_pipeline_step": 1e3 * ms / len(masks),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == "fp64" else f"f64+{prec[6:]}(fp32 acc)",
            "data": "synthetic", "gpu_launches": int(launches),
            "fbe_ms": fbe_ms, "ridc_over_fbe_time": (ms / fbe_ms) if fbe_ms else None,
            "config": {"workload": args.workload, "grid": w.n, "order": order,
                       "predictor": pred, "formal_order": order - 1 +
                       {"fbe": 1, "ark3": 3, "ark4": 4}[pred],
                       "top_level_steps": nt, "pipeline_steps": int(len(masks)),
                       "dt": w.dt, "restart_every": w.restart_every,
                       "n_refine": None if prec == "fp64" else args.n_refine,
                       "warmup_integrations": f"{args.warmup} of {warm_nt} steps",
                       "l2": "inputs larger than L2" if w.dim == 2 and S * w.n * w.n * 8 *
                             order * 4 > 129e6 else "working set fits in L2"},
            "roofline": roof,
            "kernel_ms": share,
            "rel_l2_vs_oracle": {"value": rel, "top_level_steps": k_or},
            "cpu_baseline": None if args.no_cpu else cpu,
            "clocks": clocks}
    print(json.dumps(line), flush=True)


def run_accuracy(args):
    """Accuracy of the headline workload over its whole length: the mixed path against the
    FP64 GPU path at every `--check-every` top-level steps of the 1000-step 2048^2
    Gray-Scott run, and the sensitivity envelope of the problem itself: the mixed path
    started from the initial field with every value moved by one ulp (seeded directions).
    Not a timing line; the FP64 run takes several minutes."""
    import torch

    import inputs
    from paper_1209_4297_gb300 import Integrator

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    w = inputs.gray_scott_2d(n=N, nsteps=args.nt)
    rng = np.random.default_rng(12345)
    toward = np.where(rng.random(w.u0.shape) < 0.5, -np.inf, np.inf)
    u0p = np.nextafter(w.u0, toward)
    mp = args.mixed_precision
    runs = {"mixed": (w.u0, mp), "fp64": (w.u0, "fp64"), "mixed_ulp": (u0p, mp)}
    its = {}
    for k, (u0, prec) in runs.items():
        its[k] = Integrator.from_workload(w, precision=prec, n_refine=args.n_refine,
                                          stream=stream.cuda_stream)
        its[k].set_initial(torch.from_numpy(u0).cuda())
    rows, done, t0 = [], 0, time.perf_counter()
    while done < args.nt:
        k = min(args.check_every, args.nt - done)
        for it in its.values():
            it.advance(k)
        done += k
        sol = {name: it.solution() for name, it in its.items()}
        ref = np.linalg.norm(sol["fp64"])
        rows.append({"step": done,
                     "mixed_vs_fp64": float(np.linalg.norm(sol["mixed"] - sol["fp64"]) / ref),
                     "ulp_envelope": float(np.linalg.norm(sol["mixed_ulp"] - sol["mixed"])
                                           / np.linalg.norm(sol["mixed"]))})
        print(f"# step {done}: {rows[-1]} ({time.perf_counter() - t0:.0f} s)", file=sys.stderr,
              flush=True)
    for it in its.values():
        it.close()
    line = {"metric": f"relative L2, mixed {mp[6:].upper()} ({args.n_refine} refinements) vs "
                      "FP64 GPU, 2048^2 Gray-Scott RIDC-4", "value": rows[-1]["mixed_vs_fp64"],
            "unit": "relative L2", "higher_is_better": False, "data": "synthetic",
            "config": {"workload": "gray_scott_2048_ridc4", "grid": N, "order": ORDER,
                       "top_level_steps": args.nt, "dt": 0.5, "n_refine": args.n_refine,
                       "precision": mp},
            "checkpoints": rows}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nt", type=int, default=NT, help="top-level steps per integration")
    ap.add_argument("--ref-steps", type=int, default=6)
    ap.add_argument("--fp64-steps", type=int, default=30)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--workload", default="gray_scott_2048",
                    choices=["gray_scott_2048", "ensemble", "adv_diff_1d", "adv_diff_upwind_1d",
                             "burgers_1d", "gray_scott_1024_fp64", "adv_diff_4096",
                             "accuracy_2048", "gray_scott_2048_mixed"])
    ap.add_argument("--mixed-precision", default="mixed_bf16x3",
                    choices=["mixed_bf16x3", "mixed_fp16x3"],
                    help="split form of the accuracy_2048, adv_diff_4096 and "
                         "gray_scott_2048_mixed lines (the headline line is BF16x3)")
    ap.add_argument("--order", type=int, default=None,
                    help="RIDC order of the single-workload lines (default: the workload's)")
    ap.add_argument("--n-refine", type=int, default=NREF,
                    help="refinement passes of those lines (the headline line uses 2)")
    ap.add_argument("--check-every", type=int, default=100)
    ap.add_argument("--ens-refine", type=int, default=2)
    ap.add_argument("--ens-count", type=int, default=512,
                    help="instances of the ensemble line (the configuration has 512)")
    ap.add_argument("--ens-steps", type=int, default=256,
                    help="steps of the ensemble line (the configuration has 256)")
    ap.add_argument("--oracle-steps", type=int, default=0,
                    help="top-level steps of the oracle sample of a 2D single-workload line "
                         "(0: 12 up to 1024^2, 2 above)")
    ap.add_argument("--predictor", default="fbe", choices=["fbe", "ark3", "ark4"],
                    help="level-0 predictor of the single-workload lines (Theorem 2)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "ensemble":
        return run_ensemble(args)
    if args.workload == "accuracy_2048":
        return run_accuracy(args)
    if args.workload != "gray_scott_2048":
        return run_single(args)

    import torch
    import torch.distributed as dist

    import inputs
    from paper_1209_4297_gb300 import Integrator

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.current_stream()
    w = inputs.gray_scott_2d(n=N, nsteps=args.nt)
    u0_dev = torch.from_numpy(w.u0).cuda()
    u0_host = torch.from_numpy(w.u0).pin_memory()
    out_host = torch.empty_like(u0_host).pin_memory()
    it = Integrator.from_workload(w, precision="mixed_bf16x3", n_refine=NREF,
                                  stream=stream.cuda_stream)

    def one_run():
        it.set_initial(u0_dev)
        it.advance(args.nt)

    for _ in range(args.warmup):
        one_run()
    torch.cuda.synchronize()

    # ---- timed region: device-resident inputs --------------------------------------------
    # per-kernel CUDA events on every PROF_EVERY-th pipeline step of each integration (timing
    # every launch would add about 2% to the timed region)
    it.set_profiling(PROF_EVERY)
    launches0 = it.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            one_run()
        ev1.record(stream)
        torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    launches = it.launch_count() - launches0
    ms = ev0.elapsed_time(ev1)
    stats = {k: it.kernel_stats(k) for k in ("rhs", "gemm_tc", "residual", "finalize")}
    it.set_profiling(False)
    cells = float(N * N * args.nt)
    value, ms_max = whole_job_rate(ms, cells * args.steps, device="cuda")

    # ---- end to end through the C ABI with host buffers ----------------------------------
    e2e_runs = max(1, min(args.steps, 2))
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_runs):
        it.set_initial(u0_host.numpy())
        it.advance(args.nt)
        it.solution(out_host.numpy())
    e2e_s = time.perf_counter() - t0
    e2e_val, _ = whole_job_rate(1e3 * e2e_s, cells * e2e_runs, device="cuda")
    mixed_final = out_host.numpy().copy()

    # ---- FP64 GPU form on a truncated run; accuracy of the mixed path against it ---------
    fp64 = None
    if rank == 0 and args.fp64_steps > 0:
        k = args.fp64_steps
        with Integrator.from_workload(w, precision="fp64", stream=stream.cuda_stream) as it64:
            it64.set_initial(u0_dev)
            it64.advance(2)
            torch.cuda.synchronize()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            it64.advance(k - 2)
            a1.record(stream)
            torch.cuda.synchronize()
            ref64 = it64.solution()
            fp64_rate = N * N * (k - 2) / (a0.elapsed_time(a1) * 1e-3)
        it.set_initial(u0_dev)
        it.advance(k)
        mix = it.solution()
        rel = float(np.linalg.norm(mix - ref64) / np.linalg.norm(ref64))
        fp64 = {"value": fp64_rate, "unit": UNIT, "sample": f"steps 3..{k} of the same run "
                f"(steady pipeline), FP64 DFMA fast-diagonalisation GEMMs",
                "mixed_rel_l2_vs_fp64": rel, "at_step": k}
    it.close()

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return

    peaks, peak_src = _peaks()
    # dominant kernel: the parity-split BF16x3 GEMM. One launch transforms every plane along
    # one axis as two (planes*N x N/2) x (N/2 x N/2) products, each made of 3 BF16 products:
    # 3 * planes * N^3 flop. Planes per launch come from the schedule (start-up and drain
    # steps advance fewer levels).
    n_tc, ms_tc = stats["gemm_tc"]
    planes_full = ORDER * 2
    total_gemm_flops = 0.0
    from paper_1209_4297_gb300 import schedule_plan
    masks = schedule_plan(ORDER, args.nt)
    sampled = masks[::PROF_EVERY]   # the steps whose launches were timed
    for m in sampled:
        planes = 2 * bin(int(m)).count("1")
        total_gemm_flops += 4 * (NREF + 1) * 3.0 * planes * N * N * N
    total_gemm_flops *= args.steps
    achieved_tf = total_gemm_flops / (ms_tc * 1e-3) / 1e12 if ms_tc > 0 else None
    peak_tf = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
    roof = {"bound": "tensor",
            "kernel": "gemm_sym_kernel (parity-split BF16x3 tcgen05 fast-diagonalisation)",
            "achieved": achieved_tf, "peak": peak_tf, "unit": "TFLOP/s",
            "frac": (achieved_tf / peak_tf) if achieved_tf else None,
            "peak_source": f"{peak_src} bf16_tflops_sustained",
            "flops_per_launch_full": 3.0 * planes_full * N ** 3,
            "useful_tflops": achieved_tf / 3 if achieved_tf else None,
            "dense_equivalent_tflops": 2 * achieved_tf / 3 if achieved_tf else None,
            "avg_launch_ms": ms_tc / n_tc if n_tc else None,
            "traffic": gemm_traffic(),
            "traffic_note": "DRAM bytes of one 8-plane launch (ncu); algorithmic 2.77e8",
            "timing": f"CUDA events around every launch of every {PROF_EVERY}th pipeline step "
                      "of each timed integration (on the launching stream)"}
    share = {k: {"launches": v[0], "ms": v[1]} for k, v in stats.items()}
    fp64_roof = fp64_kernel_rooflines(sampled, stats, args.steps, peaks)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "us_per_pipeline_step": 1e3 * ms_max / args.steps / len(masks),
        "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+bf16x3(fp32 acc)",
        "data": "synthetic",
        "config": {"workload": "gray_scott_2048_ridc4_mixed", "grid": N, "species": 2,
                   "order": ORDER, "top_level_steps": args.nt, "dt": 0.5, "n_refine": NREF,
                   "l2": "inputs larger than L2 (about 2.6 GB of rings and work buffers)",
                   "parallelism": f"replicas x{ws}"},
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(w.u0.nbytes),
                "d2h_bytes_per_step": int(w.u0.nbytes), "runs": e2e_runs},
        "gpu_launches": int(launches),
        "roofline": roof,
        "kernel_ms": share,
        "fp64_kernels": fp64_roof,
        "fp64_gpu": fp64,
        "clocks": clk.summary(),
    }
    if not args.no_cpu and ws == 1:
        line["cpu_baseline"] = cpu_baseline(args.ref_steps)
        line["cpu_baseline_all_cores"] = cpu_baseline(args.ref_steps, threads=os.cpu_count() or 1)
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
