#!/usr/bin/env python
"""Throughput of DNA iterations for KL-NMF on GB300 (one JSON line on stdout).

A step is one DNA iteration (H half-step then W half-step, Algorithm 1 steps 4-29) on
the workload N=4096 T=16384 R=128 (Gamma(0.3) truth scaled to mean count 2, Poisson
counts; seeded synthetic data standing in for the paper's dense datasets) in the FP32
form.  The inputs (V is 268 MB) are larger than L2, so no flush is needed between steps.
The K timed iterations are one dna_iterate call with the iteration replayed as a CUDA
graph (dna_use_graph); the dominant kernel's duration comes from event pairs around the
passes over the same K iterations launched directly, right after (events recorded inside
the graph would slow its replay), which the line also reports as direct_launches.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl dna|reference]

Under torchrun each rank solves its own independent problem (seed = rank) on its own
GPU: weak scaling with no collective on the data path; the timed region is bracketed by
barriers and the max over ranks is reported.  ``--impl reference`` times the FP64 CPU
oracle on the host cores instead (bounded column sample, scaled to the full workload).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "sec to target d_KL & DNA iters/s (BF16 vs FP32 form), % tensor peak"
UNIT = "DNA iterations/s"
SMS = 152
FP32_LANES_PER_SM = 128

ARITHMETIC = {
    ("f32", "tensor"): "float32 masters and element-wise work; each tensor-core product is "
                       "three bf16 products of hi/lo splits (x_hi y_hi + x_hi y_lo + x_lo y_hi, "
                       "about 16 significant bits per operand), float32 accumulation; float64 "
                       "cost sums",
    "f32": "float32 (CUDA-core FMA), float64 cost sums",
    "f64": "float64",
    "bf16": "bf16 tensor-core operands, float32 accumulation and masters, float64 cost sums",
}

BATCHED_DESC = ("512 problems, N ~ logU[64,2048], T ~ logU[128,8192], R ~ U{8,16,32,64}, "
                "Gamma(0.5) truth, Poisson V")

WORKLOADS = {
    "plain_large": dict(fn=workloads.plain_large, N=4096, T=16384, R=128,
                        desc="N=4096 T=16384 R=128, Gamma(0.3) truth scaled to mean 2, Poisson V"),
    "plain_small": dict(fn=workloads.plain_small, N=256, T=512, R=16,
                        desc="N=256 T=512 R=16, Gamma(0.5) truth, Poisson V"),
    "precision_large": dict(fn=workloads.precision_large, N=8192, T=32768, R=512,
                            desc="N=8192 T=32768 R=512, Gamma(0.5) W0, 70%-sparse Gamma(0.5) H0, "
                                 "V = W0 H0 + |N(0,0.01)|"),
    # the same recipe at a quarter of the size (V 268 MB, larger than L2): the case for
    # multi-pass ncu captures of the rank-512 kernels
    "precision_scaled": dict(fn=lambda seed=0: workloads.precision_large(seed, 4096, 16384, 512),
                             N=4096, T=16384, R=512,
                             desc="N=4096 T=16384 R=512, the precision_large recipe at 1/4 size"),
}


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except OSError:
        return {}


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1301_3389_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(csrc, name), "rb") as f:
                h.update(name.encode())
                h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(phase: str, workload: str):
    """DRAM bytes per launch from profiles/traffic.txt, if taken on the current sources."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    want = kernel_source_hash()
    with open(path) as f:
        for line in f:
            parts = line.split("#", 1)[0].split()
            if len(parts) == 4 and parts[0] == phase and parts[1] == workload and parts[2] == want:
                return float(parts[3])
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, local_rank: int):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        ident = vis.split(",")[local_rank].strip() if vis else str(local_rank)
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={ident}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.tmp, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.tmp.flush()
        self.tmp.seek(0)
        rows = [r.split(",") for r in self.tmp.read().splitlines() if r.strip()]
        os.unlink(self.tmp.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for name, flag in zip(names, r[5:9]):
                if flag.strip().lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def sample_columns(prob, cols: int):
    V = prob.V[:, :cols]
    H = prob.H[:, :cols]
    return V, prob.W, H


def oracle_rate(prob, cols: int, budget_s: float, min_iters: int = 1, max_iters=None):
    """FP64 oracle DNA iterations on the first ``cols`` columns; returns (iters, seconds)."""
    from oracle import dna as o
    V, W, H = sample_columns(prob, cols)
    W, H = o.normalize_w_columns(W, H)
    it, t0 = 0, time.perf_counter()
    while True:
        W, H, _, _ = o.dna_iteration(V, W, H)
        it += 1
        el = time.perf_counter() - t0
        if it >= min_iters and (el >= budget_s or (max_iters and it >= max_iters)):
            return it, el


def cpu_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_reference(args, spec, prob):
    """The FP64 CPU oracle as it stands, timed on the host cores (bounded sample)."""
    from oracle import dna as o
    cols = args.ref_cols
    V, W, H = sample_columns(prob, cols)
    W, H = o.normalize_w_columns(W, H)
    for _ in range(args.warmup):
        W, H, _, _ = o.dna_iteration(V, W, H)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        W, H, _, _ = o.dna_iteration(V, W, H)
    el = time.perf_counter() - t0
    scale = cols / spec["T"]
    value = args.steps / el * scale
    sample = (f"{args.steps} timed DNA iterations of the FP64 NumPy oracle on the first "
              f"{cols} of {spec['T']} columns; rate scaled by {cols}/{spec['T']}")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        # the measured duration of one timed step (one iteration on the column sample); the
        # full-workload figure it scales to is beside it
        "ms_per_step": el / args.steps * 1e3,
        "ms_per_step_scaled_to_full_workload": el / args.steps * 1e3 / scale,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": args.workload, "desc": spec["desc"],
                                        "sample_columns": cols},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["dna", "reference"], default="dna")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["batched", "unrolled"] + sorted(SPARSE),
                    default="plain_large")
    ap.add_argument("--dtype", choices=["f32", "f64", "bf16"], default="f32")
    ap.add_argument("--engine", choices=["auto", "simt", "tensor"], default=None,
                    help="default: tensor for f32 with R <= 512 (split bf16 products), else auto")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--cpu-budget", type=float, default=12.0, help="seconds of oracle work")
    ap.add_argument("--ref-cols", type=int, default=512)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the BF16 line and time-to-target")
    ap.add_argument("--target-iters", type=int, default=200)
    ap.add_argument("--c3-iters", type=int, default=100,
                    help="FP32 iterations that set the target at N=8192 T=32768 R=512")
    ap.add_argument("--no-c3-target", action="store_true")
    ap.add_argument("--no-mu-log", action="store_true")
    ap.add_argument("--no-sparse", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--sharded", action="store_true",
                    help="one problem split by columns over the ranks (strong scaling)")
    ap.add_argument("--log-file", default=None, help="per-iteration DNA/MU log (text)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.workload == "batched":
        return run_batched(args, world, rank, local)
    if args.workload == "unrolled":
        return run_unrolled(args, world, rank, local)
    if args.workload in SPARSE:
        return run_sparse(args, world, rank, local)
    if args.sharded:
        return run_sharded(args, world, rank, local)
    spec = WORKLOADS[args.workload]

    if args.impl == "reference":
        if rank != 0:
            return 0
        prob = spec["fn"](0)
        run_reference(args, spec, prob)
        return 0

    import torch
    import torch.distributed as dist

    import paper_1301_3389_gb300 as dna

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    prob = spec["fn"](rank)                      # independent problem per rank
    N, T, R = spec["N"], spec["T"], spec["R"]
    dev = torch.device("cuda", local)
    peaks = measured_peaks()
    if args.engine is None:
        args.engine = "tensor" if (args.dtype == "f32" and R <= 512) else "auto"
    engine_name = {"bf16": "tcgen05 (bf16 operands)", "f64": "simt"}.get(
        args.dtype, "tcgen05 (split bf16 operands, 3 products)" if args.engine == "tensor"
        else "simt")

    res = measure(dna, torch, dist, prob, args.dtype, args, world, local, peaks, clocks=True,
                  engine=args.engine)
    line = {
        "metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms_max"] / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.dtype,
        "data": "synthetic",
        "config": {"workload": args.workload, "desc": spec["desc"], "N": N, "T": T, "R": R,
                   "form": args.dtype.upper(),
                   "engine": engine_name,
                   "arithmetic": ARITHMETIC.get((args.dtype, args.engine), ARITHMETIC.get(args.dtype)),
                   "l2": "inputs larger than L2 (V is %d MB)" % (N * T * 4 // 2**20),
                   "parallelism": "independent problem per GPU" if world > 1 else "single GPU",
                   "zero_fraction": prob.meta.get("zero_fraction")},
        "gpu_launches": res["launches"],
        "roofline": res["roofline"],
        "clocks": res["clocks"],
        "kl_start": res["kl_start"], "kl_end": res["kl_end"],
        "direct_launches": res["direct"],
    }
    if args.dtype == "f32" and not args.no_forms:
        # the other forms on the same workload, and seconds to the FP32 form's target d_KL
        bf = measure(dna, torch, dist, prob, "bf16", args, world, local, peaks, clocks=False)
        line["bf16_form"] = {"value": bf["value"], "unit": UNIT,
                             "ms_per_step": bf["ms_max"] / args.steps, "roofline": bf["roofline"],
                             "gpu_launches": bf["launches"], "direct_launches": bf["direct"]}
        if args.engine == "tensor":
            sargs = argparse.Namespace(**vars(args))
            sargs.steps = max(3, min(args.steps, 20))
            sm = measure(dna, torch, dist, prob, "f32", sargs, world, local, peaks, clocks=False,
                         engine="simt")
            line["fp32_simt_form"] = {"value": sm["value"], "unit": UNIT, "steps": sargs.steps,
                                      "ms_per_step": sm["ms_max"] / sargs.steps,
                                      "roofline": sm["roofline"], "gpu_launches": sm["launches"]}
        line["time_to_target"] = time_to_target(dna, torch, prob, args.target_iters, args.engine,
                                                args.workload)
        if args.workload == "plain_large":
            # the launch-bound size N=256 T=512 R=16 (FP32 form on the tensor cores): time
            # per iteration under graph replay and with direct launches
            sspec = WORKLOADS["plain_small"]
            sprob = sspec["fn"](rank)
            sm_args = argparse.Namespace(**vars(args))
            sm_args.workload = "plain_small"
            ss = measure(dna, torch, dist, sprob, "f32", sm_args, world, local, peaks,
                         clocks=False, engine=args.engine)
            line["small_form"] = {
                "value": ss["value"], "unit": UNIT, "steps": sm_args.steps,
                "us_per_step": 1e3 * ss["ms_max"] / sm_args.steps,
                "direct_launches_us_per_step": 1e3 * ss["direct"]["ms_per_step"],
                "gpu_launches": ss["launches"],
                "config": {"workload": "plain_small", "desc": sspec["desc"], "N": sspec["N"],
                           "T": sspec["T"], "R": sspec["R"], "form": "F32",
                           "bound": "launch latency (each kernel has less than a wave of work)"}}
        if args.workload == "plain_large" and not args.no_mu_log:
            line["dna_vs_mu"] = convergence_log(dna, torch, prob, args.target_iters, args.engine,
                                                args.log_file)
            line["selection_forms"] = selection_forms(dna, torch, prob, 30)
        if args.workload == "plain_large":
            # the BF16 form at its own headline size (N=8192 T=32768 R=512), 20 iterations
            pspec = WORKLOADS["precision_large"]
            pprob = pspec["fn"](rank)
            pargs = argparse.Namespace(**vars(args))
            pargs.steps = max(3, min(args.steps, 20))
            pargs.workload = "precision_large"   # the traffic record of that workload
            pr = measure(dna, torch, dist, pprob, "bf16", pargs, world, local, peaks,
                         clocks=False)
            line["precision_form"] = {
                "value": pr["value"], "unit": UNIT, "steps": pargs.steps,
                "ms_per_step": pr["ms_max"] / pargs.steps, "roofline": pr["roofline"],
                "gpu_launches": pr["launches"], "direct_launches": pr["direct"],
                "config": {"workload": "precision_large", "desc": pspec["desc"],
                           "N": pspec["N"], "T": pspec["T"], "R": pspec["R"], "form": "BF16"}}
            if not args.no_c3_target:
                # the metric at the precision form's own size: FP32 (the split tensor-core
                # form) against BF16, to the FP32 form's d_KL after c3_iters iterations
                eng = "tensor" if pspec["R"] <= 512 else "simt"
                line["precision_form"]["time_to_target"] = time_to_target(
                    dna, torch, pprob, args.c3_iters, eng, "precision_large")
            del pprob
        if args.workload == "plain_large" and not args.no_batched:
            # the batching form: 512 uneven problems, one grouped launch per phase, CUDA graph
            bprobs = workloads.batched(512, seed=rank)
            bsteps = max(3, min(args.steps, 10))
            bres = measure_batched(dna, torch, bprobs, bsteps, args.warmup, peaks)
            line["batched_form"] = {
                "value": bsteps / (bres["ms"] / 1e3),
                "unit": "grouped DNA iterations/s (all 512 problems)",
                "ms_per_step": bres["ms"] / bsteps,
                "split_rows": bres["rows"], "gpu_launches": bres["launches"],
                "roofline": bres["roofline"],
                "config": {"workload": "batched", "desc": BATCHED_DESC, "sum_NT": bres["nt"],
                           "form": "F32", "engine": "simt grouped + CUDA graph"}}
            bb = measure_batched(dna, torch, bprobs, bsteps, args.warmup, peaks, bf16=True)
            line["batched_form"]["bf16"] = {
                "value": bsteps / (bb["ms"] / 1e3),
                "unit": "grouped DNA iterations/s (all 512 problems)",
                "ms_per_step": bb["ms"] / bsteps, "split_rows": bb["rows"],
                "pass2_units_per_cta": bb["units"], "gpu_launches": bb["launches"],
                "roofline": bb["roofline"],
                "config": {"form": "BF16", "engine": "tcgen05 grouped passes + CUDA graph"}}
            del bprobs
        if args.workload == "plain_large" and not args.no_sparse:
            sp = workloads.sparse_tdt2(rank)
            line["sparse_form"] = measure_sparse(dna, torch, sp, max(3, min(args.steps, 50)),
                                                 args.warmup, peaks)
            line["sparse_form"]["config"]["workload"] = "sparse_tdt2"

    if rank == 0 and not args.no_e2e:
        code = {"f32": dna.DNA_F32, "f64": dna.DNA_F64, "bf16": dna.DNA_BF16}[args.dtype]
        tdt = torch.float64 if args.dtype == "f64" else torch.float32
        line["e2e"] = e2e_measure(dna, torch, prob, code, tdt, N, T, R, args.e2e_steps,
                                  engine_code(dna, args.engine))
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cols = 1024
        it, el = oracle_rate(prob, cols, args.cpu_budget)
        line["cpu_baseline"] = {
            "value": it / el * cols / T, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
            "sample": f"{it} DNA iterations of the FP64 NumPy oracle on the first {cols} of {T} "
                      f"columns in {el:.1f} s, rate scaled by {cols}/{T}"}
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def max_over_ranks(torch, dist, x: float, device) -> float:
    """The largest of the ranks' values of x (the slowest rank's time)."""
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, steps: int, ms_max: float) -> float:
    """Whole-job iterations per second: every rank runs `steps` iterations of its own
    problem, and the job takes as long as the slowest rank."""
    return world * steps / (ms_max / 1e3)


def engine_code(dna, engine):
    return {"auto": dna.DNA_ENGINE_AUTO, "simt": dna.DNA_ENGINE_SIMT,
            "tensor": dna.DNA_ENGINE_TENSOR}[engine or "auto"]


def _bind(dna, torch, prob, dtype, dev, engine="auto", selection="paper"):
    code = {"f32": dna.DNA_F32, "f64": dna.DNA_F64, "bf16": dna.DNA_BF16}[dtype]
    tdt = torch.float64 if dtype == "f64" else torch.float32
    V = torch.from_numpy(prob.V).to(dev, tdt)
    W = torch.from_numpy(prob.W).to(dev, tdt)
    H = torch.from_numpy(prob.H).to(dev, tdt)
    N, T = prob.V.shape
    if dtype == "bf16":
        engine = "auto"
    ctx = dna.dna_create(N, T, prob.W.shape[1],
                         dna.make_opts(dtype=code, engine=engine_code(dna, engine)))
    dna.dna_set_stream(ctx, torch.cuda.current_stream())
    dna.dna_bind(ctx, V, W, H)
    if selection == "descent":
        dna.dna_set_selection(ctx, dna.DNA_SELECT_DESCENT)
    dna.dna_normalize(ctx, 1)                    # Algorithm 1 step 1
    return ctx, (V, W, H)


def measure(dna, torch, dist, prob, dtype, args, world, local, peaks, clocks, engine="auto"):
    """Time args.steps DNA iterations (CUDA events on the library's stream, barriers around,
    max over ranks) with per-phase event timing for the roofline of the dominant kernel."""
    dev = torch.device("cuda", local)
    N, T = prob.V.shape
    R = prob.W.shape[1]
    ctx, keep = _bind(dna, torch, prob, dtype, dev, engine)
    stream = torch.cuda.current_stream()
    kl_start = dna.dna_kl(ctx)
    # timed region: K iterations in one dna_iterate call replayed as a CUDA graph of one
    # iteration (dna_use_graph) on a stream of its own (a graph is not captured on the
    # legacy default stream)
    gstream = torch.cuda.Stream(device=dev)
    dna.dna_set_stream(ctx, gstream)
    dna.dna_use_graph(ctx, True)
    with torch.cuda.stream(gstream):
        for _ in range(args.warmup):
            dna.dna_iterate(ctx, 1)              # the first call captures the graph
        torch.cuda.synchronize()
        sampler = ClockSampler(local) if clocks else None
        if sampler:
            time.sleep(0.3)
        dna.dna_phase_times(ctx)                 # reset counters
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(gstream)
        dna.dna_iterate(ctx, args.steps)
        ev1.record(gstream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ms = ev0.elapsed_time(ev1)
        graph_phases = dna.dna_phase_times(ctx)  # launch counts of the timed region
        # the dominant kernel's duration: the same K iterations launched directly with event
        # pairs around the two passes only (events inside the graph would slow its replay)
        dna.dna_use_graph(ctx, False)
        dna.dna_profile_phases(ctx, ["pass1", "pass2"])
        d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        d0.record(gstream)
        dna.dna_iterate(ctx, args.steps)
        d1.record(gstream)
        torch.cuda.synchronize()
        direct_ms = d0.elapsed_time(d1)
        phases = dna.dna_phase_times(ctx)
        dna.dna_profile_phases(ctx, [])
        clk = sampler.stop() if sampler else None
    dna.dna_set_stream(ctx, stream)
    # phase shares from a separate, untimed pass with every phase bracketed (direct launches)
    dna.dna_profile(ctx, True)
    prof_iters = max(1, min(args.steps, 10))
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    dna.dna_iterate(ctx, prof_iters)
    e3.record(stream)
    torch.cuda.synchronize()
    prof_ms = e2.elapsed_time(e3)
    prof_phases = dna.dna_phase_times(ctx)
    dna.dna_profile(ctx, False)
    kl_end = dna.dna_kl(ctx)
    dna.dna_destroy(ctx)
    del keep
    ms_max = max_over_ranks(torch, dist, ms, dev) if world > 1 else ms
    value = job_rate(world, args.steps, ms_max)

    # roofline of the dominant kernel (largest share of the timed region)
    dom = max(("pass1", "pass2"), key=lambda p: phases[p][0])
    dom_ms, dom_launches = phases[dom]
    # one instance of each pass per half-step (an instance may be several kernel launches:
    # pass 1 of the BF16 form at R > 128 is the ratios and the contraction kernels)
    instances = 2 * args.steps
    per_launch_s = dom_ms / instances / 1e3
    flops = (6 if dom == "pass1" else 4) * R * N * T    # per launch (H or W half-step)
    alg_bytes = 4 * N * T + (8 * R * max(N, T) if dom == "pass1" else 16 * max(N, T))
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    split = dtype == "f32" and engine == "tensor"
    if split:
        # FP32-accurate products from three bf16 products each: the tensor peak available
        # to them is a third of the bf16 peak.  Executed bf16 work per launch: at R <= 128
        # pass 1 runs GEMM1 in both its A and B halves (2 x 3 x 2RNT) plus GEMM2/3
        # (2 x 3 x 2RNT); at R > 128 its ratios kernel forms Z once (3 x 2RNT) and its
        # contraction A and B (2 x 3 x 2RNT); pass 2 runs 2 x 3 x 2RNT.
        bf16_peak = float(peaks.get("bf16_tflops", 1900.0))
        fp32_peak = bf16_peak / 3.0
        p1_exec = 24 if R <= 128 else 18
        executed = (p1_exec if dom == "pass1" else 12) * R * N * T
        roof = {"bound": "tensor", "achieved": flops / per_launch_s / 1e12, "peak": fp32_peak,
                "unit": "TFLOP/s",
                "peak_source": "measured burst dense bf16 (MEASURED_PEAKS.json) / 3: three bf16 "
                               "products per FP32-accurate product (timed region well under 1 s)"}
        roof["executed_bf16_flops_per_launch"] = executed
        roof["tensor_frac_executed"] = executed / per_launch_s / 1e12 / bf16_peak
        roof["hbm_frac"] = alg_bytes / per_launch_s / 1e9 / hbm
    elif dtype == "bf16":
        tensor_peak = float(peaks.get("bf16_tflops", 1900.0))
        t_tensor = flops / (tensor_peak * 1e12)
        t_hbm = alg_bytes / (hbm * 1e9)
        if t_hbm >= t_tensor:   # the binding floor of this kernel at this size
            roof = {"bound": "hbm", "achieved": alg_bytes / per_launch_s / 1e9, "peak": hbm,
                    "unit": "GB/s", "peak_source": "measured HBM copy (MEASURED_PEAKS.json)"}
        else:
            roof = {"bound": "tensor", "achieved": flops / per_launch_s / 1e12, "peak": tensor_peak,
                    "unit": "TFLOP/s",
                    "peak_source": "measured burst dense bf16 (MEASURED_PEAKS.json; timed region "
                                   "well under 1 s)"}
        roof["tensor_frac"] = flops / per_launch_s / 1e12 / tensor_peak
        roof["hbm_frac"] = alg_bytes / per_launch_s / 1e9 / hbm
    else:
        peak = SMS * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12 if dtype == "f32" else None
        roof = {"bound": "alu", "achieved": flops / per_launch_s / 1e12, "peak": peak,
                "unit": "TFLOP/s",
                "peak_source": (f"derived: {SMS} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x "
                                f"{sm_max:.0f} MHz (max SM clock of measured)")}
    roof["frac"] = roof["achieved"] / roof["peak"] if roof.get("peak") else None
    # the whole iteration: the paper's 16 N R T useful flops (four O(NRT) products per
    # half-step) over the measured time per iteration, against the same peak
    iter_s = ms_max / args.steps / 1e3
    if split:
        iter_peak = float(peaks.get("bf16_tflops", 1900.0)) / 3.0
    elif dtype == "bf16":
        iter_peak = float(peaks.get("bf16_tflops", 1900.0))
    else:
        iter_peak = roof.get("peak") if roof["unit"] == "TFLOP/s" else None
    roof["iteration_tflops"] = 16 * R * N * T / iter_s / 1e12
    roof["iteration_frac"] = roof["iteration_tflops"] / iter_peak if iter_peak else None
    roof["kernel"] = dom
    roof["traffic"] = recorded_traffic(dom + ("_tc" if dtype == "bf16" else "_split" if split else ""),
                                       args.workload)
    roof["algorithmic_flops_per_launch"] = flops
    roof["algorithmic_bytes_per_launch"] = alg_bytes
    roof["launch_ms"] = per_launch_s * 1e3
    roof["launch_ms_source"] = ("CUDA events around each pass on the library's stream, over K "
                                "directly launched iterations right after the timed region")
    roof["kernels_per_pass"] = dom_launches / instances
    roof["phase_share"] = {p: round(prof_phases[p][0] / prof_ms, 4)
                           for p in ("pass1", "candidates", "pass2", "select", "sums", "operands")}
    roof["phase_share_note"] = (f"separate pass of {prof_iters} iterations with every phase "
                                f"bracketed by events ({prof_ms / prof_iters:.3f} ms/iteration)")
    return {"value": value, "ms_max": ms_max, "roofline": roof, "clocks": clk,
            "launches": sum(v[1] for v in graph_phases.values()), "kl_start": kl_start,
            "kl_end": kl_end,
            "direct": {"value": args.steps / (direct_ms / 1e3), "unit": UNIT,
                       "ms_per_step": direct_ms / args.steps,
                       "note": "the same iterations with every kernel launched directly and "
                               "event pairs around the two passes (the pass that gives "
                               "roofline.launch_ms), right after the timed region"}}


def run_logged(dna, torch, prob, dtype, engine, max_iters, target=None, algo="dna",
               selection="paper"):
    """Up to max_iters iterations of one form (DNA, or MU with algo="mu"), d_KL after every
    iteration.  Each iteration is timed with CUDA events on the library's stream; the d_KL
    evaluations (and the selection read-back) are outside the events.  Stops early once
    d_KL <= target.  Returns d_KL per iteration (index 0 = start), cumulative seconds, and
    for DNA the fraction of columns (H step) and rows (W step) that kept the Newton
    candidate."""
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    ctx, keep = _bind(dna, torch, prob, dtype, dev, engine, selection)
    N, T = prob.V.shape
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kls, secs, newton = [dna.dna_kl(ctx)], [0.0], []
    try:
        for _ in range(max_iters):
            torch.cuda.synchronize()
            e0.record(stream)
            if algo == "dna":
                dna.dna_iterate(ctx, 1)
            else:
                dna.mu_iterate(ctx, 1)
            e1.record(stream)
            torch.cuda.synchronize()
            secs.append(secs[-1] + e0.elapsed_time(e1) / 1e3)
            kls.append(dna.dna_kl(ctx))
            if algo == "dna":
                newton.append((float(dna.dna_get_choice(ctx, 0, T).mean()),
                               float(dna.dna_get_choice(ctx, 1, N).mean())))
            if target is not None and kls[-1] <= target:
                break
    finally:
        dna.dna_destroy(ctx)
        del keep
    return kls, secs, newton


def first_reach(kls, secs, target):
    for i, k in enumerate(kls):
        if k <= target:
            return i, secs[i]
    return None, None


def time_to_target(dna, torch, prob, iters, fp32_engine, workload):
    """Seconds and iterations for the FP32 and the BF16 form to reach the same d_KL target:
    the FP32 form's d_KL after `iters` iterations, times (1 + 1e-2).  Each form runs from
    the same start, checks d_KL after every iteration (outside the timing) and reports the
    first iteration at or below the target (the BF16 form runs at most 2 x iters)."""
    k32, s32, _ = run_logged(dna, torch, prob, "f32", fp32_engine, iters)
    target = k32[-1] * (1 + 1e-2)
    i32, t32 = first_reach(k32, s32, target)
    kb, sb, _ = run_logged(dna, torch, prob, "bf16", "auto", 2 * iters, target=target)
    ib, tb = first_reach(kb, sb, target)
    return {
        "workload": workload, "target_kl": target,
        "target_rule": f"FP32 form's d_KL after {iters} iterations x (1 + 1e-2)",
        "check": "d_KL after every iteration, outside the timed events",
        "fp32": {"engine": fp32_engine, "iterations": i32, "sec": t32,
                 "ms_per_iteration": s32[-1] / iters * 1e3, "kl_final": k32[-1]},
        "bf16": {"iterations": ib, "sec": tb, "reached": ib is not None,
                 "ms_per_iteration": sb[-1] / max(len(sb) - 1, 1) * 1e3, "kl_last": kb[-1]},
        "speedup": (t32 / tb) if (t32 and tb) else None,
    }


def selection_forms(dna, torch, prob, iters):
    """The paper's selection against descent selection (the Newton candidate against the
    starting column; one candidate's cost per half-step) in the FP32 form on the CUDA-core
    engine: time per iteration, d_KL after `iters` iterations, and the iterations and
    seconds descent needs to reach the paper rule's final d_KL."""
    kp, sp_, _ = run_logged(dna, torch, prob, "f32", "simt", iters)
    kd, sd, nd = run_logged(dna, torch, prob, "f32", "simt", 2 * iters, target=kp[-1],
                            selection="descent")
    i_d, t_d = first_reach(kd, sd, kp[-1])
    return {"engine": "simt (FP32 CUDA cores)", "iterations": iters,
            "paper": {"ms_per_iteration": sp_[-1] / iters * 1e3, "kl_final": kp[-1],
                      "sec": sp_[-1]},
            "descent": {"ms_per_iteration": sd[-1] / max(len(sd) - 1, 1) * 1e3,
                        "iterations_to_paper_final": i_d, "sec_to_paper_final": t_d,
                        "newton_fraction_last": nd[-1] if nd else None},
            "speedup_to_target": (sp_[-1] / t_d) if t_d else None}


def convergence_log(dna, torch, prob, iters, engine, log_file=None):
    """DNA and MU (eq. 11, no cost evaluation) in the FP32 form, `iters` iterations each from
    the same start, d_KL after every iteration; the iterations and seconds DNA needs to
    reach MU's final d_KL (the paper's comparison in Section 4.1), and the fraction of
    columns / rows that kept the Newton candidate."""
    kd, sd, nw = run_logged(dna, torch, prob, "f32", engine, iters, algo="dna")
    km, sm, _ = run_logged(dna, torch, prob, "f32", engine, iters, algo="mu")
    target = km[-1]
    i_d, t_d = first_reach(kd, sd, target)
    marks = [i for i in (0, 1, 2, 3, 5, 10, 20, 50, 100, 150, 200, 300, 500) if i <= iters]
    if log_file:
        with open(log_file, "w") as f:
            f.write("iteration kl_dna sec_dna kl_mu sec_mu newton_frac_H newton_frac_W\n")
            for i in range(iters + 1):
                nh, nww = nw[i - 1] if i > 0 else (float("nan"), float("nan"))
                f.write(f"{i} {kd[i]:.10e} {sd[i]:.6e} {km[i]:.10e} {sm[i]:.6e} {nh:.4f} {nww:.4f}\n")
    return {
        "iterations": iters, "engine": engine,
        "target": "MU's d_KL after %d iterations" % iters,
        "dna_iterations_to_mu_final": i_d, "dna_sec_to_mu_final": t_d, "mu_sec": sm[-1],
        "iteration_ratio": (iters / i_d) if i_d else None,
        "time_ratio": (sm[-1] / t_d) if t_d else None,
        "ms_per_iteration": {"dna": sd[-1] / iters * 1e3, "mu": sm[-1] / iters * 1e3},
        "kl_at": {str(i): {"dna": kd[i], "mu": km[i]} for i in marks},
        "newton_fraction_at": {str(i): {"H": nw[i - 1][0], "W": nw[i - 1][1]}
                               for i in marks if i > 0},
    }


SPARSE = {
    "sparse_tdt2": (workloads.sparse_tdt2, "36771 x 10212 term counts, 0.35 % non-zeros, R=64 "
                    "(TDT2's shape), synthetic"),
    "sparse_newsgroup": (workloads.sparse_newsgroup, "61188 x 18774 term counts, 0.2 % "
                         "non-zeros, R=64 (Newsgroup's shape), synthetic"),
}


def measure_sparse(dna, torch, sp, steps, warmup, peaks, dtype="f32"):
    """DNA iterations of the sparse-V form (CSR V, passes over the non-zeros only): CUDA
    events around `steps` iterations in one dna_iterate call, events around the two passes
    for the dominant kernel's roofline (algorithmic bytes: the index and value of every
    non-zero, the column pointers and each factor once, per pass)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    tdt = torch.float64 if dtype == "f64" else torch.float32
    rp = torch.from_numpy(sp.row_ptr).to(dev)
    ci = torch.from_numpy(sp.col_idx).to(dev)
    vals = torch.from_numpy(sp.vals).to(dev, tdt)
    W = torch.from_numpy(sp.W).to(dev, tdt)
    H = torch.from_numpy(sp.H).to(dev, tdt)
    R = sp.W.shape[1]
    code = dna.DNA_F64 if dtype == "f64" else dna.DNA_F32
    ctx = dna.dna_create_sparse(sp.N, sp.T, R, sp.nnz, dna.make_opts(dtype=code))
    stream = torch.cuda.current_stream()
    try:
        dna.dna_set_stream(ctx, stream)
        dna.dna_bind_csr(ctx, rp, ci, vals, W, H)
        dna.dna_normalize(ctx, 1)
        kl0 = dna.dna_kl(ctx)
        dna.dna_iterate(ctx, warmup)
        dna.dna_profile_phases(ctx, ["pass1", "pass2"])
        dna.dna_phase_times(ctx)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dna.dna_iterate(ctx, steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        ph = dna.dna_phase_times(ctx)
        # phase shares from a separate, untimed pass with every phase bracketed
        dna.dna_profile(ctx, True)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        dna.dna_iterate(ctx, 10)
        f1.record(stream)
        torch.cuda.synchronize()
        pms = f0.elapsed_time(f1)
        pph = dna.dna_phase_times(ctx)
        dna.dna_profile(ctx, False)
        kl1 = dna.dna_kl(ctx)
    finally:
        dna.dna_destroy(ctx)
    es = 8 if dtype == "f64" else 4
    # per pass: each non-zero's index (4 B) and value, the O + 1 pointers, both factors once
    bytes_h = sp.nnz * (4 + es) + (sp.T + 1) * 8 + es * R * (sp.N + sp.T)
    bytes_w = sp.nnz * (4 + es) + (sp.N + 1) * 8 + es * R * (sp.N + sp.T)
    dom = max(("pass1", "pass2"), key=lambda p: ph[p][0])
    dom_ms, dom_n = ph[dom]
    per_launch = dom_ms / max(dom_n, 1) / 1e3
    alg = (bytes_h + bytes_w) / 2                  # average over the H and W views
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    it_bytes = 2 * (bytes_h + bytes_w)             # two passes per view
    return {
        "value": steps / (ms / 1e3), "unit": UNIT, "steps": steps, "ms_per_step": ms / steps,
        "config": {"N": sp.N, "T": sp.T, "R": R, "nnz": sp.nnz, "density": sp.nnz / (sp.N * sp.T),
                   "form": dtype.upper(), "engine": "simt sparse (warp per column / row)"},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": alg / per_launch / 1e9,
                     "peak": hbm, "unit": "GB/s", "frac": alg / per_launch / 1e9 / hbm,
                     "traffic": None, "algorithmic_bytes_per_launch": alg,
                     "launch_ms": per_launch * 1e3,
                     "iteration_hbm_frac": it_bytes / (ms / steps / 1e3) / 1e9 / hbm,
                     "note": "the rows of the fixed factor gathered per non-zero are served "
                             "by L2 and not counted; the passes are bound by those gathers",
                     "phase_share": {p: round(pph[p][0] / pms, 4) for p in
                                     ("pass1", "candidates", "pass2", "select", "sums", "operands")}},
        "kl_start": kl0, "kl_end": kl1,
    }


def run_sparse(args, world, rank, local):
    """The sparse-V form on a synthetic term-count workload (one line)."""
    import torch

    import paper_1301_3389_gb300 as dna
    torch.cuda.set_device(local)
    fn, desc = SPARSE[args.workload]
    sp = fn(rank)
    peaks = measured_peaks()
    clocks = ClockSampler(local)
    time.sleep(0.3)
    res = measure_sparse(dna, torch, sp, args.steps, args.warmup, peaks, args.dtype)
    clk = clocks.stop()
    line = {"metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.dtype, "data": "synthetic",
            "config": dict(res["config"], workload=args.workload, desc=desc,
                           l2="factors and indices fit L2; no flush (steady-state iterations)"),
            "roofline": res["roofline"], "clocks": clk,
            "kl_start": res["kl_start"], "kl_end": res["kl_end"]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_sharded(args, world, rank, local):
    """One problem (the workload) split by columns over the ranks (strong scaling): each
    rank's GPU holds V[:, block], H[:, block] and a copy of W; the exchanges of the W
    half-step and of the normalisations are NCCL all-reduces (paper_1301_3389_gb300.sharded).
    A step is one DNA iteration of the whole problem."""
    import torch
    import torch.distributed as dist

    import paper_1301_3389_gb300 as dna
    from paper_1301_3389_gb300.sharded import ShardedDNA
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    spec = WORKLOADS[args.workload]
    prob = spec["fn"](0)                                # the same problem on every rank
    N, T, R = spec["N"], spec["T"], spec["R"]
    cuts = np.linspace(0, T, world + 1).astype(int)
    a, b = int(cuts[rank]), int(cuts[rank + 1])
    V = torch.from_numpy(np.ascontiguousarray(prob.V[:, a:b])).to(dev)
    W = torch.from_numpy(prob.W).to(dev)
    H = torch.from_numpy(np.ascontiguousarray(prob.H[:, a:b])).to(dev)
    del prob
    engine = args.engine or ("tensor" if R <= 512 else "auto")
    ctx = dna.dna_create(N, b - a, R, dna.make_opts(dtype=dna.DNA_F32, engine=engine_code(dna, engine)))
    stream = torch.cuda.current_stream()
    dna.dna_set_stream(ctx, stream)
    dna.dna_bind(ctx, V, W, H)
    dna.dna_normalize(ctx, 1)
    sh = ShardedDNA([ctx], N, R, torch.float32, all_reduce=dist.all_reduce if world > 1 else None)
    kl0 = sh.kl()
    sh.iterate(args.warmup)
    clocks = ClockSampler(local) if rank == 0 else None
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sh.iterate(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop() if clocks else None
    ms_max = max_over_ranks(torch, dist, ms, dev) if world > 1 else ms
    kl1 = sh.kl()
    dna.dna_destroy(ctx)
    if world > 1:
        dist.destroy_process_group()
    line = {"metric": METRIC, "value": args.steps / (ms_max / 1e3), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "desc": spec["desc"], "N": N, "T": T, "R": R,
                       "parallelism": f"columns split over {world} GPUs, W replicated, NCCL "
                                      "all-reduce of the W half-step's sums",
                       "engine": engine, "l2": "inputs larger than L2"},
            "clocks": clk, "kl_start": kl0, "kl_end": kl1}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def measure_batched(dna, torch, probs, steps, warmup, peaks, bf16=False):
    """Grouped DNA iterations of all problems (every phase one grouped launch, the
    iteration replayed as a CUDA graph, tile sizes autotuned), timed with CUDA events.
    bf16: the BF16 form (passes on the tensor cores), else FP32 on the CUDA cores."""
    dev = torch.device("cuda", torch.cuda.current_device())
    V = [torch.from_numpy(p.V).to(dev) for p in probs]
    W = [torch.from_numpy(p.W).to(dev) for p in probs]
    H = [torch.from_numpy(p.H).to(dev) for p in probs]
    shapes = [p.shape for p in probs]
    opts = dna.make_opts(dtype=dna.DNA_BF16) if bf16 else None
    g = dna.dna_group_create([s[0] for s in shapes], [s[1] for s in shapes], [s[2] for s in shapes],
                             opts)
    stream = torch.cuda.current_stream()
    try:
        dna.dna_group_set_stream(g, stream)
        dna.dna_group_bind(g, V, W, H)
        dna.dna_group_normalize(g, 1)
        rows = dna.dna_group_autotune(g, 2)
        _, units = dna.dna_group_tile_config(g)
        dna.dna_group_use_graph(g, True)
        kl0 = dna.dna_group_kl(g, len(probs))
        dna.dna_group_iterate(g, warmup)
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        # the timed iterations form the profiler range (ncu --profile-from-start off)
        torch.cuda.profiler.start()
        ev0.record(stream)
        dna.dna_group_iterate(g, steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        ms = ev0.elapsed_time(ev1)
        kl1 = dna.dna_group_kl(g, len(probs))
        # BF16: plus the first H half-step's operands, written once per dna_group_iterate call
        launches = dna.dna_group_launches_per_iteration(g) * steps + (1 if bf16 else 0)
    finally:
        dna.dna_group_destroy(g)
    nt = sum(s[0] * s[1] for s in shapes)
    alg_bytes = 4 * 4 * nt          # V read by both passes of both half-steps, float32
    flops = sum(20 * s[2] * s[0] * s[1] for s in shapes)   # 10 R flop per element per half-step
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    step_s = ms / steps / 1e3
    achieved = flops / step_s / 1e12
    out = {"ms": ms, "rows": rows, "units": units, "launches": launches, "kl0": kl0, "kl1": kl1,
           "nt": nt}
    if bf16:
        # at R <= 64 the grouped passes read far more bytes than the tensor pipe needs time
        # for: HBM bound (V, float32, 16 bytes per element per iteration)
        tensor = float(peaks.get("bf16_tflops", 1900.0))
        out["roofline"] = {"bound": "hbm", "kernel": "whole grouped iteration",
                           "achieved": alg_bytes / step_s / 1e9, "peak": hbm, "unit": "GB/s",
                           "frac": alg_bytes / step_s / 1e9 / hbm, "traffic": None,
                           "algorithmic_flops_per_step": flops,
                           "algorithmic_bytes_per_step": alg_bytes,
                           "tensor_frac": achieved / tensor,
                           "peak_source": "measured HBM copy (MEASURED_PEAKS.json)"}
    else:
        alu = SMS * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
        out["roofline"] = {"bound": "alu", "kernel": "whole grouped iteration",
                           "achieved": achieved, "peak": alu, "unit": "TFLOP/s",
                           "frac": achieved / alu, "traffic": None,
                           "algorithmic_flops_per_step": flops,
                           "algorithmic_bytes_per_step": alg_bytes,
                           "hbm_frac": alg_bytes / step_s / 1e9 / hbm,
                           "peak_source": (f"derived: {SMS} SMs x {FP32_LANES_PER_SM} FP32 lanes "
                                           f"x 2 flop x {sm_max:.0f} MHz")}
    return out


def run_batched(args, world, rank, local):
    """The batching form: one step = one DNA iteration of all 512 problems, every phase one
    grouped launch, the iteration replayed as a CUDA graph, split sizes autotuned."""
    import torch
    import torch.distributed as dist

    import paper_1301_3389_gb300 as dna
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    probs = workloads.batched(512, seed=rank)
    dev = torch.device("cuda", local)
    clocks = ClockSampler(local)
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    bf16 = args.dtype == "bf16"
    res = measure_batched(dna, torch, probs, args.steps, args.warmup, measured_peaks(), bf16=bf16)
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms_max = max_over_ranks(torch, dist, res["ms"], dev) if world > 1 else res["ms"]
    if world > 1:
        dist.destroy_process_group()
    value = job_rate(world, args.steps, ms_max)
    line = {
        "metric": METRIC, "value": value, "unit": "grouped DNA iterations/s (all 512 problems)",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16" if bf16 else "f32", "data": "synthetic",
        "config": {"workload": "batched", "desc": BATCHED_DESC, "problems": len(probs),
                   "sum_NT": res["nt"], "form": "BF16" if bf16 else "F32",
                   "engine": ("tcgen05 grouped passes + CUDA graph" if bf16
                              else "simt grouped + CUDA graph"),
                   "split_rows": res["rows"], "pass2_units_per_cta": res["units"],
                   "l2": "inputs larger than L2 (V totals %d MB)" % (res["nt"] * 4 >> 20)},
        "gpu_launches": res["launches"],
        "roofline": res["roofline"],
        "clocks": clk,
        "kl_sum_start": float(np.sum(res["kl0"])), "kl_sum_end": float(np.sum(res["kl1"])),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


UNROLLED_K, UNROLLED_EVERY = 20, 5


def run_unrolled(args, world, rank, local):
    """The differentiation form: one step = the K = 20 unrolled DNA H-solve with W held by
    the solve (checkpoints every 5 steps), the loss d_KL(V, W H_K) + (mu / 2) |H_K|^2 and
    its backward pass to V, W and H0, through the autograd wrappers (N=1024 T=4096 R=64).
    With the F32 form the line also gives the relative error of each gradient against the
    F64 form's (the F64 form is tested against the FP64 reference to 1e-8)."""
    import torch
    import torch.distributed as dist

    from paper_1301_3389_gb300.autograd import KLDiv, UnrolledDNAH
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    prob = workloads.diff_form(rank)
    dev = torch.device("cuda", local)
    dt = torch.float64 if args.dtype == "f64" else torch.float32
    N, T = prob.V.shape
    R = prob.W.shape[1]
    mu = 1e-3 * float(prob.V.mean()) / float(prob.H.mean()) ** 2
    def leaves(dtype):
        return tuple(torch.from_numpy(x).to(dev, dtype).requires_grad_(True)
                     for x in (prob.V, prob.W, prob.H))

    V, W, H0 = leaves(dt)

    def step(V=V, W=W, H0=H0):
        V.grad = W.grad = H0.grad = None
        HK = UnrolledDNAH.apply(V, W, H0, UNROLLED_K, UNROLLED_EVERY)
        loss = KLDiv.apply(V, W, HK) + 0.5 * mu * (HK.double() ** 2).sum()
        loss.backward()
        return loss

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    # V is 16 MB: L2 is flushed (a 256 MB write) before every step, outside its events
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        loss = step()
        ev1.record(stream)
        torch.cuda.synchronize()
        ms += ev0.elapsed_time(ev1)
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms_max = max_over_ranks(torch, dist, ms, dev) if world > 1 else ms
    if world > 1:
        dist.destroy_process_group()
    value = job_rate(world, args.steps, ms_max)
    accuracy = None
    if dt == torch.float32:
        # the F32 gradients of the last timed step against the F64 form's, same inputs
        g32 = [x.grad.double() for x in (V, W, H0)]
        V64, W64, H64 = leaves(torch.float64)
        step(V64, W64, H64)
        torch.cuda.synchronize()
        accuracy = {"reference": "F64 form of the same solve and loss",
                    "K": UNROLLED_K}
        for name, g, x in zip(("dL/dV", "dL/dW", "dL/dH0"), g32, (V64, W64, H64)):
            accuracy[name] = float(torch.linalg.norm(g - x.grad) / torch.linalg.norm(x.grad))
    # forward: K H half-steps of about 10 R N T flop; backward: the segments' recomputed
    # steps (K - K / every) plus K adjoint steps of about 10 R N T each (z recomputed, the
    # two z-tiles P1, P2 and H-bar's product) and K W-gradient steps of about 12 R N T (z,
    # P1, P2 recomputed, then the three sums over o), and d_KL's backward (4 R N T)
    K, ev = UNROLLED_K, UNROLLED_EVERY
    flops = (K + (K - K // ev) + K) * 10 * R * N * T + K * 12 * R * N * T + 4 * R * N * T
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    if dt == torch.float64:
        alu, alu_src = 1.25, "nominal GB300 FP64 rate (1.25 TFLOP/s)"
    else:
        alu = SMS * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
        alu_src = f"derived: {SMS} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x {sm_max:.0f} MHz"
    step_s = ms_max / args.steps / 1e3
    achieved = flops / step_s / 1e12
    line = {
        "metric": METRIC, "value": value,
        "unit": "unrolled-solve forward + backward steps/s (K = 20 H half-steps)",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if dt == torch.float64 else "f32",
        "data": "synthetic",
        "config": {"workload": "unrolled", "N": N, "T": T, "R": R, "K": K, "every": ev,
                   "mu": mu, "engine": "CUDA cores (F32 / F64 forms)",
                   "l2": "L2 flushed (256 MB write) before each step, outside the timed events"},
        "roofline": {"bound": "alu", "kernel": "whole forward + backward step",
                     "achieved": achieved, "peak": alu, "unit": "TFLOP/s",
                     "frac": achieved / alu, "traffic": None,
                     "algorithmic_flops_per_step": flops, "peak_source": alu_src},
        "clocks": clk, "loss": float(loss),
        "gradients": "V, W and H0",
    }
    if accuracy is not None:
        line["accuracy_rel_fro"] = accuracy
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def e2e_measure(dna, torch, prob, code, tdt, N, T, R, steps, engine=0):
    """Iterations/s through dna_run_host on pinned host buffers: each step copies V, W, H
    in, runs one DNA iteration, and copies W, H and d_KL out."""
    Vh = torch.from_numpy(prob.V).to(tdt).pin_memory()
    Wh = torch.from_numpy(prob.W).to(tdt).pin_memory()
    Hh = torch.from_numpy(prob.H).to(tdt).pin_memory()
    ctx = dna.dna_create(N, T, R, dna.make_opts(dtype=code, engine=engine))
    try:
        dna.dna_set_stream(ctx, torch.cuda.current_stream())
        for _ in range(3):
            dna.dna_run_host(ctx, Vh, Wh, Hh, 1)
        t0 = time.perf_counter()
        for _ in range(steps):
            dna.dna_run_host(ctx, Vh, Wh, Hh, 1)
        el = time.perf_counter() - t0
    finally:
        dna.dna_destroy(ctx)
    es = Vh.element_size()
    return {"value": steps / el, "unit": UNIT,
            "h2d_bytes_per_step": es * (N * T + N * R + R * T),
            "d2h_bytes_per_step": es * (N * R + R * T) + 8}


if __name__ == "__main__":
    sys.exit(main())
