#!/usr/bin/env python3
"""Benchmark of the QBX hot path on GB300.

One step = the three on-surface operator applies (S, D, grad S, two-sided) of
the full-size starfish workload: r(t) = 1 + 0.25 cos 5t, 256 panels x 16
targets (4096), 16384 oversampled sources, k = 20, p = 12, interior and
exterior centres (8192), CN(0,1) density (seed 2).  Metric: QBX
centre x source x order terms per second (term = (centre, source, l),
l in [-p, p], x rhs), whole job.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

--impl reference times the CPU oracle (the plain FP64 restatement of the
method) on the host cores, on a bounded sample of targets per step.
Under torchrun (N > 1) every rank runs an independent replica of the workload
on its own GPU (no data-path collective; weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "QBX center·source·order terms/s"
# FP64 ALU peak of the dominant kernel's pipe: 152 SMs x 2 FP64 FMA lanes per
# SM per clock (4 flops) x 2.07 GHz maximum SM clock (nominal 1.25 TFLOP/s).
FP64_PEAK_GFLOPS = 152 * 4 * 2.07
# Algorithmic FP64 flop model per (centre, source) pair of the fused apply
# (FMA = 2 flops), counted from the algorithm the kernel runs, real k:
#   one operator alone: 100 flops of pair set-up (distance, H0, H1) + 16 per
#   order (S) or 24 per order (D, grad S), + 8 per extra right-hand side;
#   S, D and grad S in one pass (shared set-up and recurrences): 180 flops of
#   set-up + 35 per order (S 5, D 7, grad S 10, shared recurrences 13),
#   + 32 per extra right-hand side.
FLOPS_PAIR = {"S": (100, 16), "D": (100, 24), "GRAD_S": (100, 24)}


def flops_per_pair(op, p, nrhs=1):
    a, b = FLOPS_PAIR[op]
    return a + b * p + 8 * (nrhs - 1)


def flops_per_pair_ops(ops, p, nrhs=1):
    if len(ops) == 1:
        return flops_per_pair(ops[0], p, nrhs)
    if set(ops) == {"S", "D", "GRAD_S"}:
        return 180 + 35 * p + 32 * (nrhs - 1)
    # other subsets: shared set-up once, each operator's own products
    per = {"S": 5, "D": 7, "GRAD_S": 10}
    acc = {"S": 8, "D": 8, "GRAD_S": 16}
    rec = 7 + (4 if "D" in ops else 0) + (2 if "GRAD_S" in ops else 0)
    return 140 + sum(acc[o] for o in ops) + p * (rec + sum(per[o] for o in ops)) + \
        (nrhs - 1) * sum(acc[o] for o in ops)


# DRAM bytes (read + write) of one launch of the fused S + D + grad S kernel
# on the full-size starfish workload, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum); valid only for the kernel
# sources it was taken with, identified by their hash.
TRAFFIC = {"27706399748d3043": 1.667e6}   # profiles/k_apply_fused_S_D_gradS_starfish_M256_dram.md
KERNEL_SOURCES = ["qbx_apply_impl.cuh", "qbx_device.cuh", "special_tables.h", "qbx_apply_real.cu"]
GROUP_SOURCES = ["qbx_group_impl.cuh", "qbx_apply_impl.cuh", "qbx_device.cuh", "special_tables.h"]
# Hardware-counted FP64 operations per (centre, source) pair, 2 DFMA + DMUL +
# DADD from ncu's smsp__sass_thread_inst_executed_op_{dfma,dmul,dadd}_pred_on
# counters divided by the pairs of the captured launch, for the kernel
# sources with the given hash (profiles/fp64_counts_fused_M128_and_group_batch4.md).
HW_FP64_PER_PAIR = {"27706399748d3043": 434.9}         # fused S + D + grad S, p = 12, one rhs
HW_FP64_PER_PAIR_GROUP = {"5b690bb633cedf23": 732.9}   # group kernel, S + D, p = 10, 32 rhs
# sm__pipe_fp64_cycles_active (of peak) over the active and the elapsed
# cycles, from the same captures (fused: 128-panel starfish, one wave;
# group: the first 4 curves of the batch)
HW_FP64_PIPE = {"27706399748d3043": (0.922, 0.880)}
HW_FP64_PIPE_GROUP = {"5b690bb633cedf23": (0.949, 0.926)}
# the fused S + D + grad S apply at the complex wavenumber 20 + 1i (same
# capture set-up: 128-panel starfish, p = 12, one rhs)
HW_FP64_PER_PAIR_CPLX = {"27706399748d3043": 726.4}
HW_FP64_PIPE_CPLX = {"27706399748d3043": (0.923, 0.878)}


def source_hash(names=KERNEL_SOURCES):
    """Hash of the kernel sources' code (comments and blank space removed, so
    that only a change of the code itself invalidates a recorded count)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_1207_4461_gb300", "csrc", name)) as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def kernel_source_hash():
    return source_hash(KERNEL_SOURCES)


def hw_roofline(ops_per_pair, pairs, seconds, pipe=None):
    if ops_per_pair is None:
        return None
    a = pairs * ops_per_pair / seconds / 1e9
    out = {"fp64_ops_per_pair": ops_per_pair, "achieved": a, "frac": a / FP64_PEAK_GFLOPS,
           "unit": "GFLOP/s", "source": "ncu FP64 instruction counters (2 DFMA + DMUL + DADD) of the same "
                                        "kernel sources, per pair, x pairs / measured kernel time"}
    if pipe is not None:
        out["fp64_pipe_busy"] = {"of_active_cycles": pipe[0], "of_elapsed_cycles": pipe[1],
                                 "source": "ncu sm__pipe_fp64_cycles_active of the same kernel sources"}
    return out


def kernel_traffic(wl, args):
    if args.separate or args.panels or args.ops or args.k:
        return None
    return TRAFFIC.get(kernel_source_hash())


def max_over_ranks(x, torch, device, world):
    """The largest of the ranks' values (the job's time under replicas); x
    itself for one rank.  One all_reduce(MAX) of a float64 on `device`."""
    if world <= 1:
        return x
    t = torch.tensor([x], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, units_per_rank, ms):
    """Whole-job throughput: `world` replicas, each `units_per_rank` units in
    `ms` (the max over ranks)."""
    return world * units_per_rank / (ms * 1e-3)


def env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_sample(wl, n_targets, reps=1):
    """Time the CPU oracle on `n_targets` sampled targets of the workload (all
    three operators, both sides).  Returns (terms, seconds, threads)."""
    import oracle
    go = oracle.geometry(wl.curve, wl.curve.edges(wl.M), wl.q_tgt, wl.q_src)
    dens = wl.dens(go["t_tgt"])
    rng = np.random.default_rng(0)
    sel = np.sort(rng.choice(wl.n_tgt, n_targets, replace=False))
    ops = {"S": oracle.OP_S, "D": oracle.OP_D, "GRAD_S": oracle.OP_GRAD_S}
    t0 = time.perf_counter()
    for _ in range(reps):
        for name in wl.ops:
            oracle.apply(go, ops[name], oracle.SIDE_TWO, 0, wl.k, wl.p, dens, sel=sel)
    dt = time.perf_counter() - t0
    sides = 2 if wl.sides == "two" else 1
    terms = reps * len(wl.ops) * n_targets * sides * wl.n_src * (2 * wl.p + 1) * wl.nrhs
    return terms, dt, oracle.num_threads()


def run_reference(args, wl):
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    n = args.ref_sample
    for _ in range(args.warmup):
        oracle_sample(wl, max(4, n // 8))
    times, terms = [], 0
    for _ in range(args.steps):
        t, dt, cores = oracle_sample(wl, n)
        times.append(dt)
        terms += t
    total = sum(times)
    value = terms / total
    sample = (f"{n} of {wl.n_tgt} targets per step (both sides, S, D and grad S, all "
              f"{wl.n_src} sources), CPU: {cpu_model()}")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "terms/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(wl, args),
            "cpu_baseline": {"value": value, "unit": "terms/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "terms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def config_dict(wl, args):
    return {"workload": f"starfish r=1+0.25cos5t, M={wl.M} panels x {wl.q_tgt} targets "
                        f"({wl.n_tgt}), {wl.n_src} sources (4x), k={wl.k:g}, p={wl.p}, "
                        f"two-sided centres ({wl.n_ctr}), ops S+D+gradS, CN(0,1) density seed {wl.seed}",
            "n_tgt": wl.n_tgt, "n_src": wl.n_src, "n_ctr": wl.n_ctr,
            "k": wl.k if isinstance(wl.k, float) else str(wl.k), "p": wl.p,
            "nrhs": wl.nrhs, "terms_per_step": len(wl.ops) * wl.terms_per_op(),
            "l2": "flushed between timed steps (256 MiB write outside the event pair)",
            "parallelism": "replicas" if args.gpus > 1 else "single",
            "call": "qbx_apply per operator" if args.separate else "qbx_apply_ops (one pass for all operators)"}


def run_gpu(args, wl):
    import torch
    import paper_1207_4461_gb300 as qbx

    rank, world, local = env_rank()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    ops = {"S": qbx.OP_S, "D": qbx.OP_D, "GRAD_S": qbx.OP_GRAD_S}
    codes = [ops[n] for n in wl.ops]
    ncomp = sum(2 if n == "GRAD_S" else 1 for n in wl.ops)
    plan = qbx.Plan(wl.q_tgt, wl.q_src, n_src=wl.n_src, n_ctr=wl.n_ctr, ncoef=ncomp, nrhs=wl.nrhs)
    g = qbx.qbx_geometry(plan, wl.curve, wl.curve.edges(wl.M))
    dens_np = wl.dens(g.t_tgt)
    dens = torch.as_tensor(dens_np, device=dev).contiguous()
    outs = {ops[n]: torch.empty((wl.n_tgt, 2, wl.nrhs) if n == "GRAD_S" else (wl.n_tgt, wl.nrhs),
                                dtype=torch.complex128, device=dev) for n in wl.ops}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step(d, kernel_ms=None):
        if args.separate:
            for c in codes:
                qbx.qbx_apply(plan, g, c, qbx.SIDE_TWO, 0, wl.k, wl.p, d, out_on=outs[c])
                if kernel_ms is not None:
                    kernel_ms[-1] += qbx.qbx_plan_kernel_ms(plan)
        else:  # all operators in one pass over the pairs
            qbx.qbx_apply_ops(plan, g, codes, qbx.SIDE_TWO, 0, wl.k, wl.p, d, out=outs)
            if kernel_ms is not None:
                kernel_ms[-1] += qbx.qbx_plan_kernel_ms(plan)

    if args.min_waves:
        qbx.qbx_plan_set_min_waves(plan, args.min_waves)
    qbx.qbx_plan_set_timing(plan, True)   # events around the pair-sum kernel of every call
    for _ in range(args.warmup):
        step(dens)
    torch.cuda.synchronize()
    qbx.qbx_sync_status(plan)

    # ---- device-timed region: K steps, events per step, L2 flushed between steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0])
                          if os.environ.get("CUDA_VISIBLE_DEVICES", "").isdigit() else local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    kernel_ms = []
    for s in range(args.steps):
        flush.fill_(s & 0xFF)
        ev[s][0].record(stream)
        kernel_ms.append(0.0)
        step(dens, kernel_ms)
        ev[s][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    kern_ms = sum(kernel_ms) / len(kernel_ms)
    steps_ms = [a.elapsed_time(b) for a, b in ev]
    step_ms = sum(steps_ms) / args.steps
    qbx.qbx_sync_status(plan)
    step_ms = max_over_ranks(step_ms, torch, dev, world)
    terms_step = len(wl.ops) * wl.terms_per_op()
    value = job_rate(world, terms_step, step_ms)

    # roofline of the dominant kernel (the fused apply): algorithmic flops / duration
    pairs = wl.n_ctr * wl.n_src
    if args.separate:
        fpp = sum(flops_per_pair(n, wl.p, wl.nrhs) for n in wl.ops)
        kname = "k_apply_fused, one launch per operator"
    else:
        fpp = flops_per_pair_ops(list(wl.ops), wl.p, wl.nrhs)
        kname = "k_apply_fused, operators " + "+".join(wl.ops) + " in one pass"
    achieved = pairs * fpp / (kern_ms * 1e-3) / 1e9
    hw = None
    if not (args.separate or args.panels or args.ops or args.k):
        hw = hw_roofline(HW_FP64_PER_PAIR.get(kernel_source_hash()), pairs, kern_ms * 1e-3,
                         HW_FP64_PIPE.get(kernel_source_hash()))
    # headline: hardware-counted FP64 flops (2 DFMA + DMUL + DADD per pair from
    # ncu, for these kernel sources) per second against the FP64 peak; the
    # algorithmic model beside it; the model alone when no count matches
    roofline = {"bound": "alu", "achieved": hw["achieved"] if hw else achieved, "peak": FP64_PEAK_GFLOPS,
                "unit": "GFLOP/s", "frac": hw["frac"] if hw else achieved / FP64_PEAK_GFLOPS,
                "basis": "ncu-counted FP64 flops per pair" if hw else "algorithmic flop model per pair",
                "traffic": kernel_traffic(wl, args),
                "kernel": kname, "kernel_ms": kern_ms,
                "timing": "CUDA events recorded by the library around the kernel launch(es) of every "
                          "timed call, on the launching stream",
                "flops_per_pair": hw["fp64_ops_per_pair"] if hw else fpp,
                "peak_basis": "152 SMs x 4 FP64 flop/clk x 2.07 GHz",
                "model": {"flops_per_pair": fpp, "achieved": achieved, "frac": achieved / FP64_PEAK_GFLOPS},
                "hw": hw}

    # ---- end to end through the public API with host buffers (pinned)
    h_dens = torch.from_numpy(dens_np).pin_memory()
    h_outs = {c: torch.empty(outs[c].shape, dtype=torch.complex128).pin_memory() for c in outs}
    d_dens = torch.empty_like(dens)
    h2d = h_dens.numel() * 16
    d2h = sum(o.numel() * 16 for o in h_outs.values())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(2):
        d_dens.copy_(h_dens, non_blocking=True)
        step(d_dens)
    torch.cuda.synchronize()
    e2e_ms = 0.0
    for s in range(args.steps):
        flush.fill_(s & 0xFF)
        e0.record(stream)
        d_dens.copy_(h_dens, non_blocking=True)
        step(d_dens)
        for c in outs:
            h_outs[c].copy_(outs[c], non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_ms += e0.elapsed_time(e1)
    e2e_ms = max_over_ranks(e2e_ms / args.steps, torch, dev, world)
    e2e = {"value": job_rate(world, terms_step, e2e_ms), "unit": "terms/s",
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms}

    launches = (3 * len(wl.ops)) if args.separate else (2 + len(wl.ops))   # upsample, fused, finish(es)
    line = {"metric": METRIC, "value": value, "unit": "terms/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config_dict(wl, args),
            "roofline": roofline, "e2e": e2e, "clocks": clk,
            "gpu_launches": args.steps * launches,
            "targets_per_s": world * len(wl.ops) * wl.n_tgt * wl.nrhs / (step_ms * 1e-3),
            "pairs_per_s": world * len(wl.ops) * pairs / (step_ms * 1e-3)}
    if rank == 0 and not args.separate:
        line["near_only"] = run_local_compare(args, qbx, torch, plan, g, codes, wl, dens, outs, flush, stream,
                                              step_ms)
    if rank == 0 and not args.panels and not args.separate and not args.k and not args.ops:
        line["complex_k"] = run_complex_k(args, qbx, torch, plan, g, codes, wl, dens, outs, flush, stream)
    if rank == 0 and not args.no_batch and not args.panels:
        line["batched"] = run_batch_compare(args, qbx, torch, small=False)
        line["batched_small"] = run_batch_compare(args, qbx, torch, small=True)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        terms, dt, cores = oracle_sample(wl, args.cpu_sample)
        import oracle
        oracle.set_num_threads(1)   # the same oracle on one core, smaller sample
        terms1, dt1, _ = oracle_sample(wl, max(8, args.cpu_sample // 24))
        oracle.set_num_threads(cores)
        line["cpu_baseline"] = {"value": terms / dt, "unit": "terms/s", "cores": cores, "kind": "oracle",
                                "single_core_value": terms1 / dt1,
                                "single_core_sample": f"{max(8, args.cpu_sample // 24)} targets, {dt1:.1f} s",
                                "sample": f"{args.cpu_sample} of {wl.n_tgt} targets, both sides, S, D and "
                                          f"grad S, all {wl.n_src} sources; CPU: {cpu_model()}",
                                "seconds": dt}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_local_compare(args, qbx, torch, plan, g, codes, wl, dens, outs, flush, stream, global_ms, eta=8.0):
    """Near-only QBX (qbx_apply_local, sources beyond eta r by the smooth rule
    at the target) on the same step: time per step and the largest relative
    difference from the global apply's outputs (not the benchmark metric)."""
    loc = {c: torch.empty_like(outs[c]) for c in outs}
    for _ in range(2):
        qbx.qbx_apply_ops(plan, g, codes, qbx.SIDE_TWO, 0, wl.k, wl.p, dens, out=loc, eta=eta)
    torch.cuda.synchronize()
    tot = 0.0
    steps = max(1, min(args.steps, 5))
    for s in range(steps):
        flush.fill_(s & 0xFF)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        qbx.qbx_apply_ops(plan, g, codes, qbx.SIDE_TWO, 0, wl.k, wl.p, dens, out=loc, eta=eta)
        e1.record(stream)
        e1.synchronize()
        tot += e0.elapsed_time(e1)
    ms = tot / steps
    qbx.qbx_apply_ops(plan, g, codes, qbx.SIDE_TWO, 0, wl.k, wl.p, dens, out=outs)
    diff = max((torch.abs(loc[c] - outs[c]).max() / torch.abs(outs[c]).max()).item() for c in outs)
    return {"eta": eta, "ms_per_step": ms, "speedup_vs_global": global_ms / ms, "max_rel_diff_vs_global": diff,
            "call": "qbx_apply_local (sources with |x_s - c| >= eta r by the smooth rule at the target)"}


def batch_workload(small):
    """The batched comparison's workloads: the 64 random curves of 16..512
    panels, or 256 small ones (16..48 panels), where every per-curve launch
    fills a small part of the GPU."""
    if small:
        return W.BatchWorkload("fourier-batch-256-small", 256, 10, 32, 4, m_lo=16, m_hi=48)
    return W.cfg3()


def spread(xs):
    xs = sorted(xs)
    n = len(xs)
    med = xs[n // 2] if n % 2 else 0.5 * (xs[n // 2 - 1] + xs[n // 2])
    return {"median": med, "min": xs[0], "max": xs[-1], "samples": n}


def run_complex_k(args, qbx, torch, plan, g, codes, wl, dens, outs, flush, stream, k=20.0 + 1.0j):
    """The same step at the complex wavenumber k = 20 + 1i (Im k > 0: complex
    J_l, complex recurrences, H0 and H1 from the amplitude table of the ray
    z = k rho): time per step, kernel time and the counted-flop roofline (not
    the benchmark metric)."""
    out = {c: torch.empty_like(outs[c]) for c in outs}
    for _ in range(2):
        qbx.qbx_apply_ops(plan, g, codes, qbx.SIDE_TWO, 0, k, wl.p, dens, out=out)
    torch.cuda.synchronize()
    qbx.qbx_sync_status(plan)
    steps = max(3, min(args.steps, 5))
    tot, kern = 0.0, 0.0
    for s in range(steps):
        flush.fill_(s & 0xFF)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        qbx.qbx_apply_ops(plan, g, codes, qbx.SIDE_TWO, 0, k, wl.p, dens, out=out)
        e1.record(stream)
        e1.synchronize()
        tot += e0.elapsed_time(e1)
        kern += qbx.qbx_plan_kernel_ms(plan)
    qbx.qbx_sync_status(plan)
    ms, kms = tot / steps, kern / steps
    pairs = wl.n_ctr * wl.n_src
    terms = len(wl.ops) * wl.terms_per_op()
    return {"k": str(k), "ms_per_step": ms, "kernel_ms": kms, "terms_per_s": terms / (ms * 1e-3), "steps": steps,
            "roofline_hw": hw_roofline(HW_FP64_PER_PAIR_CPLX.get(kernel_source_hash()), pairs, kms * 1e-3,
                                       HW_FP64_PIPE_CPLX.get(kernel_source_hash())),
            "parity": "tests/test_gpu_parity.py::test_apply_full_size_complex_k (the oracle at 256 targets, "
                      "both sides, S, D and grad S, <= 1e-11 per output array)"}


def run_batch_compare(args, qbx, torch, small=None):
    """Many random curves (p = 10, 32 densities, S and D): one batched launch
    (CUDA graph) against one qbx_apply_ops call per curve, the two arms
    alternating step by step (>= 10 timed steps each, L2 flushed before every
    step), reported as median, min and max.  Returns the figures for the JSON
    line."""
    bw = batch_workload(args.batch_small if small is None else small)
    insts = bw.instances()
    if args.batch_curves:
        insts = insts[:args.batch_curves]
    Mmax = max(M for _, M, _ in insts)
    plan = qbx.Plan(bw.q_tgt, bw.q_src, n_src=bw.q_src * Mmax, n_ctr=bw.q_tgt * Mmax, ncoef=2, nrhs=bw.nrhs)
    geoms = [qbx.qbx_geometry(plan, c, c.edges(M)) for c, M, _ in insts]
    dens = [torch.as_tensor(bw.dens(i, g.n_tgt), device="cuda").contiguous() for i, g in enumerate(geoms)]
    ks = [k for _, _, k in insts]
    batch = qbx.Batch(plan, geoms, ks, bw.p, (qbx.OP_S, qbx.OP_D), qbx.SIDE_INT, 0, dens)
    model_cfg = batch.info()
    t_tune = time.perf_counter()
    batch.tune()   # outside the timed region: measured choice of items and rhs grouping
    t_tune = time.perf_counter() - t_tune
    tuned_cfg = batch.info()
    outs = [{o: torch.empty_like(batch.out[i][o]) for o in (qbx.OP_S, qbx.OP_D)} for i in range(len(geoms))]
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def per_instance():
        for i, g in enumerate(geoms):
            qbx.qbx_apply_ops(plan, g, (qbx.OP_S, qbx.OP_D), qbx.SIDE_INT, 0, ks[i], bw.p, dens[i], out=outs[i])

    def one(fn, s):
        flush.fill_(s & 0xFF)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1)

    batch.apply()
    per_instance()
    torch.cuda.synchronize()
    steps = max(10, args.batch_steps)
    t_batch, t_inst = [], []
    for s in range(steps):   # alternate the arms so that drifts of the clock hit both
        if s % 2 == 0:
            t_batch.append(one(batch.apply, 2 * s))
            t_inst.append(one(per_instance, 2 * s + 1))
        else:
            t_inst.append(one(per_instance, 2 * s))
            t_batch.append(one(batch.apply, 2 * s + 1))
    batch.status()
    qbx.qbx_sync_status(plan)
    sb, si = spread(t_batch), spread(t_inst)
    ms_batch, ms_inst = sb["median"], si["median"]
    # the same batch with near-only QBX (eta = 8), then back to the global apply
    batch.set_eta(8.0)
    batch.apply()
    ms_near = one(batch.apply, 0)
    batch.set_eta(0.0)
    batch.status()
    pairs = sum(g.n_tgt * g.n_src for g in geoms)
    terms = pairs * (2 * bw.p + 1) * bw.nrhs * 2
    fpp = flops_per_pair_ops(["S", "D"], bw.p, bw.nrhs)
    achieved = pairs * fpp / (ms_batch * 1e-3) / 1e9
    full64 = not args.batch_curves and bw.n_inst == 64
    return {"workload": f"{len(insts)} random Fourier curves r=1+sum_{{m<=8}}(a_m cos mt+b_m sin mt), "
                        f"a,b~U(-0.04,0.04), M~U{{{bw.m_lo}..{bw.m_hi}}} x 16 targets, 4x sources, k~U(1,40), "
                        f"p=10, 32 CN(0,1) densities, interior, S and D (seed {bw.seed})",
            "pairs": pairs, "terms_per_step": terms, "steps": steps,
            "timing": "arms alternating step by step, CUDA events on the launching stream, L2 flushed before "
                      "each step; medians",
            "batched_ms": ms_batch, "per_instance_ms": ms_inst,
            "batched_ms_spread": sb, "per_instance_ms_spread": si,
            "ranges_overlap": not (sb["max"] < si["min"] or si["max"] < sb["min"]),
            "batched_terms_per_s": terms / (ms_batch * 1e-3),
            "per_instance_terms_per_s": terms / (ms_inst * 1e-3),
            "speedup": ms_inst / ms_batch,
            "near_only_batched_ms": ms_near,
            "items": {"model": dict(zip(("rhs_per_warp", "src_chunk", "items", "ctas"), model_cfg)),
                      "tuned": dict(zip(("rhs_per_warp", "src_chunk", "items", "ctas"), tuned_cfg)),
                      "tune_s": t_tune},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                         "frac": achieved / FP64_PEAK_GFLOPS, "flops_per_pair": fpp,
                         "kernel": "k_apply_group (persistent, longest-first items, CUDA graph)",
                         "timing": "whole graph (oversampling, group kernel, finishing) per apply",
                         "hw": None if not full64 else hw_roofline(
                             HW_FP64_PER_PAIR_GROUP.get(source_hash(GROUP_SOURCES)), pairs, ms_batch * 1e-3,
                             HW_FP64_PIPE_GROUP.get(source_hash(GROUP_SOURCES)))}}


def run_solve(args):
    """Exterior sound-soft scattering (Sec. 4.2): (1/2 + D - i eta S) mu = f,
    eta = k, two-sided D and S, on the paper's teardrop with 1008 panels
    equispaced in t and the panel on each side of the corner bisected 8
    times (1024 panels, 16384 targets, 65536 sources, 32768 centres), k = 30,
    p = 14, f = -e^{i k d_m . x} for 64 plane waves d_m = (cos 2 pi m/64,
    sin 2 pi m/64), GMRES(restart) on the device to 1e-10.  Prints one JSON
    line (not the benchmark metric): solve time, matvecs, time per matvec,
    residuals (GMRES's and one recomputed by a separate apply); the same
    solve on the assembled matrix."""
    import torch
    import paper_1207_4461_gb300 as qbx
    torch.cuda.set_device(0)
    k, p, nrhs, m_base, levels = 30.0, 14, 64, args.solve_base, 8
    # the paper's teardrop (about 115 degrees), or the right-angle one with the
    # admissible radius (r = h/2 lowered where a source enters the disk)
    cur = W.teardrop(args.corner90)
    edges = W.dyadic_edges(m_base, levels)
    M = len(edges) - 1
    plan = qbx.Plan(16, 64, n_src=64 * M, n_ctr=32 * M, ncoef=2, nrhs=nrhs)
    rule = qbx.RADIUS_ADMISSIBLE if args.corner90 else qbx.RADIUS_H
    g = qbx.qbx_geometry(plan, cur, edges, rule=rule)
    if args.assemble_only:   # the assembly kernel alone (profiling), after one warm-up call
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        A = qbx.qbx_assemble_cfie(plan, g, k, k, p)
        torch.cuda.synchronize()
        e0.record()
        A = qbx.qbx_assemble_cfie(plan, g, k, k, p)
        e1.record()
        e1.synchronize()
        qbx.qbx_sync_status(plan)
        print(json.dumps({"assemble": f"teardrop, {m_base}+{2 * levels} panels, k=30, p=14", "n_tgt": g.n_tgt,
                          "n_src": g.n_src, "ms": e0.elapsed_time(e1),
                          "pairs": 2 * g.n_tgt * g.n_src}))
        return 0
    tx, ty = g["tgt_x"], g["tgt_y"]
    ang = 2 * math.pi * torch.arange(nrhs, dtype=torch.float64, device="cuda") / nrhs
    f = -torch.exp(1j * k * (tx[:, None] * torch.cos(ang)[None, :] + ty[:, None] * torch.sin(ang)[None, :]))
    f = f.contiguous()
    # one matvec alone (the combined field (D - i eta S) mu two-sided, 64 rhs:
    # qbx_apply_cfie, as the solve calls it), timed after a warm-up
    d = f.clone()
    out_c = torch.empty_like(d)
    qbx.qbx_plan_set_timing(plan, True)
    qbx.qbx_apply_cfie(plan, g, k, k, p, d, out=out_c)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    qbx.qbx_apply_cfie(plan, g, k, k, p, d, out=out_c)
    e1.record()
    e1.synchronize()
    mv_ms = e0.elapsed_time(e1)
    mv_kernel_ms = qbx.qbx_plan_kernel_ms(plan)
    qbx.qbx_plan_set_timing(plan, False)
    if args.solve_matvec_only:   # profiling: the matvec alone
        print(json.dumps({"matvec": "(D - i eta S) two-sided, 64 rhs (the solve's matvec, qbx_apply_cfie)",
                          "n_tgt": g.n_tgt, "n_src": g.n_src, "matvec_ms": mv_ms, "matvec_kernel_ms": mv_kernel_ms}))
        return 0
    clocks = ClockSampler(0)
    clocks.start()
    e0.record()
    mu, its, res = qbx.qbx_solve_exterior_dirichlet(plan, g, k, k, p, f, tol=1e-10, restart=args.solve_restart,
                                                     maxiter=args.solve_maxiter, raise_on_noconv=False)
    e1.record()
    e1.synchronize()
    clk = clocks.stop()
    solve_ms = e0.elapsed_time(e1)
    qbx.qbx_sync_status(plan)
    # the same solve on the assembled matrix (one qbx_matmul_cm product per matvec)
    e0.record()
    A = qbx.qbx_assemble_cfie(plan, g, k, k, p)
    e1.record()
    e1.synchronize()
    asm_ms = e0.elapsed_time(e1)
    # twice (the first call also queries the product's split)
    asm_ms_calls = []
    for _ in range(2):
        e0.record()
        mu_a, its_a, res_a = qbx.qbx_solve_exterior_dirichlet(plan, g, k, k, p, f, tol=1e-10,
                                                             restart=args.solve_restart, maxiter=args.solve_maxiter,
                                                             raise_on_noconv=False, A=A)
        e1.record()
        e1.synchronize()
        asm_ms_calls.append(e0.elapsed_time(e1))
    asm_solve_ms = asm_ms_calls[-1]
    mu_diff = (torch.abs(mu_a - mu).max() / torch.abs(mu).max()).item()
    prod_ms = time_matmul(torch, qbx, A, f, 3)["own_ms"]
    del A
    # the residual recomputed by one more apply of both operators to mu: in
    # GMRES's norm (sqrt-weighted 2-norm per rhs, relative to f) and pointwise
    # (max |r| / max |f|, largest at the refined corner panels); the oracle's
    # residual at sampled targets is a test
    sd = {qbx.OP_S: torch.empty_like(mu), qbx.OP_D: torch.empty_like(mu)}
    qbx.qbx_apply_ops(plan, g, (qbx.OP_S, qbx.OP_D), qbx.SIDE_TWO, 0, k, p, mu.contiguous(), out=sd)
    r = 0.5 * mu + sd[qbx.OP_D] - 1j * k * sd[qbx.OP_S] - f
    sw = torch.sqrt(g["tgt_w"])[:, None]
    resid_w = (torch.linalg.norm(sw * r, dim=0) / torch.linalg.norm(sw * f, dim=0)).max().item()
    resid_apply = (torch.abs(r).max() / torch.abs(f).max()).item()
    pairs = 2 * g.n_tgt * g.n_src
    curve_name = ("teardrop with a 90-degree corner, admissible radius (r = h/2 lowered to the largest "
                  "source-free disk)" if args.corner90 else "paper's teardrop (2 atan(pi/2), about 115 degrees)")
    line = {"solve": f"exterior sound-soft, {curve_name}, {m_base}+16 panels (dyadic toward the corner), "
                     "k=30, p=14, eta=k, 64 plane waves, two-sided D and S, GMRES on the device",
            "n_tgt": g.n_tgt, "n_src": g.n_src, "n_ctr": 2 * g.n_tgt, "nrhs": nrhs,
            "restart": args.solve_restart, "tol": 1e-10, "matvecs": its,
            "converged": bool(np.all(res <= 1e-10)), "max_resid": float(np.max(res)),
            "solve_s": solve_ms * 1e-3, "matvec_ms": mv_ms, "matvec_kernel_ms": mv_kernel_ms,
            "pairs_per_matvec": pairs,
            "terms_per_s_matvec": 2 * pairs * (2 * p + 1) * nrhs / (mv_ms * 1e-3),
            "resid_by_apply_weighted_l2": resid_w, "resid_by_apply_pointwise": resid_apply,
            "assembled": {"assembly_s": asm_ms * 1e-3, "solve_s": asm_solve_ms * 1e-3,
                          "first_solve_call_s": asm_ms_calls[0] * 1e-3, "matvecs": its_a,
                          "max_resid": float(np.max(res_a)), "max_rel_diff_vs_matrix_free": mu_diff,
                          "matrix_bytes": 16 * g.n_tgt * g.n_tgt,
                          "product_ms": prod_ms,
                          "outside_products_s": asm_solve_ms * 1e-3 - (its_a + 2) * prod_ms * 1e-3,
                          "outside_products_note": "solve time less (matvecs + restart residuals) x one product: "
                                                   "Arnoldi kernels, launches and the one host wait per cycle",
                          "call": "qbx_assemble_cfie + qbx_solve_exterior_dirichlet_assembled (qbx_matmul_cm "
                                  "products; one Arnoldi step as a CUDA graph, Givens and residual tests on the "
                                  "device)"},
            "clocks": clk}
    print(json.dumps(line))
    return 0


def time_matmul(torch, qbx, A, x, reps, library=False):
    """qbx_matmul_cm on the column-major matrix A ([n][n] tensor, A(i, j) at
    [j][i]) and x [n][nrhs]: mean time of `reps` calls after a warm-up call
    (CUDA events); with library=True also torch's complex matmul of the same
    product (cuBLAS ZGEMM), as the library reference."""
    n = A.shape[0]
    work = torch.empty(max(qbx.lib().qbx_matmul_cm_work_bytes(n, x.shape[1]), 16), dtype=torch.uint8, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    y = qbx.qbx_matmul_cm(A, x, work)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        y = qbx.qbx_matmul_cm(A, x, work)
    e1.record()
    e1.synchronize()
    out = {"own_ms": e0.elapsed_time(e1) / reps}
    if library:
        ref = A.T @ x
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            ref = A.T @ x
        e1.record()
        e1.synchronize()
        out["library_ms"] = e0.elapsed_time(e1) / reps
        out["max_rel_diff_vs_library"] = ((y - ref).abs().max() / ref.abs().max()).item()
    return out


def run_matmul(args):
    """The assembled solve's product alone: y = A x, A a seeded random complex
    n x n matrix (column-major), x n x 64, by qbx_matmul_cm (FP64, three real
    products per complex multiply-add) and by torch's matmul (cuBLAS ZGEMM)
    for reference.  Prints one JSON line (not the benchmark metric)."""
    import torch
    import paper_1207_4461_gb300 as qbx
    torch.cuda.set_device(0)
    n, nrhs = args.matmul_n, 64
    g = torch.Generator(device="cuda").manual_seed(7)
    A = torch.randn((n, n), dtype=torch.complex128, device="cuda", generator=g)
    x = torch.randn((n, nrhs), dtype=torch.complex128, device="cuda", generator=g)
    clocks = ClockSampler(0)
    clocks.start()
    t = time_matmul(torch, qbx, A, x, args.steps, library=True)
    clk = clocks.stop()
    flops = 3 * 2 * n * n * nrhs   # three real products per complex multiply-add
    line = {"matmul": f"y = A x, A {n} x {n} complex (column-major), x {n} x {nrhs}, FP64", "n": n, "nrhs": nrhs,
            "steps": args.steps, **t, "own_gflops": flops / (t["own_ms"] * 1e-3) / 1e9,
            "own_frac_of_fp64_peak": flops / (t["own_ms"] * 1e-3) / 1e9 / FP64_PEAK_GFLOPS,
            "flops_model": "3 real products x 2 flops per complex multiply-add", "clocks": clk}
    print(json.dumps(line))
    return 0


def fourier_curve_samples(torch, coef, t):
    """gamma = r(t)(cos t, sin t), r = a0 + sum_{m=1..8} a_m cos mt + b_m sin mt,
    coef = (a0, a1..a8, b1..b8) as a torch tensor: gamma and gamma' at the
    parameters t (torch), differentiable in coef."""
    m = torch.arange(1, 9, dtype=torch.float64, device=coef.device)
    cm, sm = torch.cos(t[:, None] * m), torch.sin(t[:, None] * m)
    r = coef[0] + cm @ coef[1:9] + sm @ coef[9:17]
    dr = (-sm * m) @ coef[1:9] + (cm * m) @ coef[9:17]
    c, s_ = torch.cos(t), torch.sin(t)
    return torch.stack([r * c, r * s_], -1), torch.stack([dr * c - r * s_, dr * s_ + r * c], -1)


def run_adjoint(args):
    """Shape-optimisation workload (loss ||S sigma - g||^2, interior centres):
    the starfish r = 1 + 0.25 cos 5t written as 17 Fourier coefficients of
    r(t), 128 panels (2048 targets, 8192 sources), k = 10, p = 10,
    sigma = cos 3t + 0.5 i sin t, g = e^{i k x}.  Times, with CUDA events and
    the L2 flushed before every call: the forward S apply, the density
    adjoint (transposed sweep), the shape adjoint, and one whole
    loss-and-gradient step through autograd (curve samples from the
    coefficients, geometry, S apply, backward to the 17 coefficients and the
    density).  Prints one JSON line (not the benchmark metric)."""
    import torch
    import paper_1207_4461_gb300 as qbx
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    M, k, p, side = 128, 10.0, 10, qbx.SIDE_INT
    edges = np.linspace(0.0, 2 * np.pi, M + 1)
    plan = qbx.Plan(16, 64, workspace_bytes=qbx.qbx_shape_adjoint_workspace_bytes(M, 16, 64, p, 1))
    tt = torch.as_tensor(qbx.panel_nodes(edges, 16), device=dev)
    ts = torch.as_tensor(qbx.panel_nodes(edges, 64), device=dev)
    c0 = torch.zeros(17, dtype=torch.float64, device=dev)
    c0[0], c0[5] = 1.0, 0.25
    gt, dgt = fourier_curve_samples(torch, c0, tt)
    gs, dgs = fourier_curve_samples(torch, c0, ts)
    g = qbx.qbx_geometry_samples(plan, edges, gt.contiguous(), dgt.contiguous(), gs.contiguous(), dgs.contiguous())
    sig = torch.as_tensor(W.density_cfg1(tt.cpu().numpy()), device=dev).reshape(-1, 1).contiguous()
    target = torch.exp(1j * k * gt[:, 0]).reshape(-1, 1)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(args.steps):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.median(ms)

    u = qbx.qbx_apply(plan, g, qbx.OP_S, side, 0, k, p, sig)
    gout = (2 * (u - target)).contiguous()
    clocks = ClockSampler(0)
    clocks.start()
    t_fwd = timed(lambda: qbx.qbx_apply(plan, g, qbx.OP_S, side, 0, k, p, sig))
    t_adj = timed(lambda: qbx.qbx_apply_adjoint(plan, g, qbx.OP_S, side, 0, k, p, gout))
    t_shape = timed(lambda: qbx.qbx_apply_shape_adjoint(plan, g, side, k, p, sig, gout))

    def loss_and_grad():
        coef = c0.clone().requires_grad_(True)
        s = sig.clone().requires_grad_(True)
        a, da = fourier_curve_samples(torch, coef, tt)
        b, db = fourier_curve_samples(torch, coef, ts)
        v = qbx.apply_s_shape_autograd(plan, edges, a, da, b, db, s, side, k, p)
        L = (torch.abs(v - torch.exp(1j * k * a[:, 0]).reshape(-1, 1)) ** 2).sum()
        L.backward()
        return coef.grad, s.grad

    t_step = timed(loss_and_grad)
    # D: forward, shape adjoint and a loss-and-gradient step of ||D mu - g||^2
    ud = qbx.qbx_apply(plan, g, qbx.OP_D, side, 0, k, p, sig)
    goutd = (2 * (ud - target)).contiguous()
    t_fwd_d = timed(lambda: qbx.qbx_apply(plan, g, qbx.OP_D, side, 0, k, p, sig))
    t_shape_d = timed(lambda: qbx.qbx_apply_shape_adjoint(plan, g, side, k, p, sig, goutd, op=qbx.OP_D))

    def loss_and_grad_d():
        coef = c0.clone().requires_grad_(True)
        s = sig.clone().requires_grad_(True)
        a, da = fourier_curve_samples(torch, coef, tt)
        b, db = fourier_curve_samples(torch, coef, ts)
        v = qbx.apply_d_shape_autograd(plan, edges, a, da, b, db, s, side, 0, k, p)
        L = (torch.abs(v - torch.exp(1j * k * a[:, 0]).reshape(-1, 1)) ** 2).sum()
        L.backward()
        return coef.grad, s.grad

    t_step_d = timed(loss_and_grad_d)
    clk = clocks.stop()
    qbx.qbx_sync_status(plan)
    # the adjoint identity Re <S sigma, y> = Re <sigma, S^H y> for a random y
    y = torch.as_tensor(W.complex_gaussian(7, g.n_tgt).reshape(-1, 1), device=dev)
    lhs = torch.vdot(y.flatten(), u.flatten())
    rhs = torch.vdot(qbx.qbx_apply_adjoint(plan, g, qbx.OP_S, side, 0, k, p, y).flatten(), sig.flatten())
    ident = (torch.abs(lhs - rhs) / (torch.abs(y).sum() * torch.abs(u).max())).item()
    n_ctr, n_src = g.n_tgt, g.n_src
    terms = n_ctr * n_src * (2 * p + 1)
    print(json.dumps({
        "adjoint": "shape-optimisation loss ||S sigma - g||^2, starfish r = 1 + 0.25 cos 5t as 17 Fourier "
                   "coefficients, 128 panels (2048 targets, 8192 sources, 2048 interior centres), k=10, p=10",
        "n_tgt": g.n_tgt, "n_src": g.n_src, "n_ctr": n_ctr, "p": p, "k": k, "steps": args.steps,
        "warmup": args.warmup, "l2": "flushed before every timed call (256 MiB write outside the event pair)",
        "forward_ms": t_fwd, "density_adjoint_ms": t_adj, "shape_adjoint_ms": t_shape,
        "loss_and_gradient_step_ms": t_step,
        "forward_terms_per_s": terms / (t_fwd * 1e-3),
        "density_adjoint_terms_per_s": terms / (t_adj * 1e-3),
        "density_adjoint_over_forward": t_adj / t_fwd, "shape_adjoint_over_forward": t_shape / t_fwd,
        "adjoint_identity_relerr": ident,
        "d": {"loss": "||D mu - g||^2, interior limit, same curve and density", "forward_ms": t_fwd_d,
              "shape_adjoint_ms": t_shape_d, "shape_adjoint_over_forward": t_shape_d / t_fwd_d,
              "loss_and_gradient_step_ms": t_step_d,
              "calls": "qbx_apply (D), qbx_apply_shape_adjoint_d, QBXShapeD through autograd"},
        "calls": "qbx_apply (S), qbx_apply_adjoint (S), qbx_apply_shape_adjoint; step: qbx_geometry_samples + "
                 "qbx_apply forward, qbx_apply_adjoint + qbx_apply_shape_adjoint backward, torch for r(t)",
        "clocks": clk}))
    return 0


def run_variants(args):
    """The operator variants on the full-size starfish workload (256 panels,
    4096 targets, 16384 sources, both sides, k = 20, p = 12, one CN(0,1)
    density): the tangential dipole R (D's sums with the source tangents),
    grad D (storage-free), S + D + grad S on centres at r = c sqrt(h)
    (c = 0.08, about the h/2 radius at this panel size), and near-only
    S + D + grad S (eta = 8), beside the global S + D + grad S step; then
    S, D and grad S through stored coefficients (form, then evaluate),
    S + D + grad S at the complex wavenumber 20 + 1i, and S + D + grad S for
    32 right-hand sides (the group kernel), global and near-only.  CUDA events per call, L2 flushed
    before every timed call.  Prints one JSON line (not the benchmark
    metric)."""
    import torch
    import paper_1207_4461_gb300 as qbx
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    wl = W.cfg2()
    if args.panels:
        wl.M = args.panels
    plan = qbx.Plan(wl.q_tgt, wl.q_src, n_src=wl.n_src, n_ctr=wl.n_ctr, ncoef=2 * wl.p + 1, nrhs=1)
    g = qbx.qbx_geometry(plan, wl.curve, wl.curve.edges(wl.M))
    g_sq = qbx.qbx_geometry(plan, wl.curve, wl.curve.edges(wl.M), 0.08, qbx.RADIUS_SQRT_H)
    dens = torch.as_tensor(wl.dens(g.t_tgt), device=dev).contiguous()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    ops3 = (qbx.OP_S, qbx.OP_D, qbx.OP_GRAD_S)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(args.steps):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.median(ms)

    clocks = ClockSampler(0)
    clocks.start()
    t = {
        "S+D+grad S": timed(lambda: qbx.qbx_apply_ops(plan, g, ops3, qbx.SIDE_TWO, 0, wl.k, wl.p, dens)),
        "R": timed(lambda: qbx.qbx_apply(plan, g, qbx.OP_R, qbx.SIDE_TWO, 0, wl.k, wl.p, dens)),
        "grad D (PV)": timed(lambda: qbx.qbx_apply(plan, g, qbx.OP_GRAD_D, qbx.SIDE_TWO, qbx.LIMIT_PV, wl.k, wl.p,
                                                 dens)),
        "S+D+grad S, r = 0.08 sqrt(h)": timed(lambda: qbx.qbx_apply_ops(plan, g_sq, ops3, qbx.SIDE_TWO, 0, wl.k,
                                                                        wl.p, dens)),
        "S+D+grad S, near-only eta = 8": timed(lambda: qbx.qbx_apply_ops(plan, g, ops3, qbx.SIDE_TWO, 0, wl.k, wl.p,
                                                                         dens, eta=8.0)),
    }
    # the same three operators through stored coefficients (Sec. 3.3 as
    # written: form alpha for S and for D, then evaluate S, D and grad S;
    # raw expansion values, without the finishing step)
    KS, KD = qbx.OP_S, qbx.OP_D

    def stored():
        wdn = qbx.qbx_upsample(plan, g, dens)
        a_s = qbx.qbx_form_locals(plan, g, KS, qbx.SIDE_TWO, wl.k, wl.p, wdn)
        a_d = qbx.qbx_form_locals(plan, g, KD, qbx.SIDE_TWO, wl.k, wl.p, wdn)
        qbx.qbx_eval_locals(plan, g, qbx.SIDE_TWO, wl.k, wl.p, a_s, qbx.VALUE)
        qbx.qbx_eval_locals(plan, g, qbx.SIDE_TWO, wl.k, wl.p, a_d, qbx.VALUE)
        qbx.qbx_eval_locals(plan, g, qbx.SIDE_TWO, wl.k, wl.p, a_s, qbx.GRAD)
    t["S, D, grad S via stored coefficients (form + eval)"] = timed(stored)
    # complex wavenumber (absorbing medium): the amplitude table of the ray z = k rho
    kc = complex(wl.k, 1.0)
    t["S+D+grad S, k = 20 + 1i"] = timed(lambda: qbx.qbx_apply_ops(plan, g, ops3, qbx.SIDE_TWO, 0, kc, wl.p, dens))
    # 32 rhs of one density: the group kernel, global and near-only
    plan32 = qbx.Plan(wl.q_tgt, wl.q_src, n_src=wl.n_src, n_ctr=wl.n_ctr, ncoef=4, nrhs=32)
    g32 = qbx.qbx_geometry(plan32, wl.curve, wl.curve.edges(wl.M))
    d32 = torch.as_tensor(W.complex_gaussian(5, g32.n_tgt * 32).reshape(g32.n_tgt, 32), device=dev)
    t["S+D+grad S, 32 rhs"] = timed(lambda: qbx.qbx_apply_ops(plan32, g32, ops3, qbx.SIDE_TWO, 0, wl.k, wl.p, d32))
    t["S+D+grad S, 32 rhs, near-only eta = 8"] = timed(
        lambda: qbx.qbx_apply_ops(plan32, g32, ops3, qbx.SIDE_TWO, 0, wl.k, wl.p, d32, eta=8.0))
    t["S+D+grad S, 32 rhs, k = 20 + 1i"] = timed(
        lambda: qbx.qbx_apply_ops(plan32, g32, ops3, qbx.SIDE_TWO, 0, kc, wl.p, d32))
    qbx.qbx_sync_status(plan32)
    # near-only accuracy against speed: eta sweep (largest relative difference from the global apply)
    glob = qbx.qbx_apply_ops(plan, g, ops3, qbx.SIDE_TWO, 0, wl.k, wl.p, dens)
    glob = {o: v.clone() for o, v in glob.items()}
    eta_sweep = {}
    for eta in (3.0, 5.0, 8.0, 12.0):
        ms = timed(lambda: qbx.qbx_apply_ops(plan, g, ops3, qbx.SIDE_TWO, 0, wl.k, wl.p, dens, eta=eta))
        loc = qbx.qbx_apply_ops(plan, g, ops3, qbx.SIDE_TWO, 0, wl.k, wl.p, dens, eta=eta)
        diff = max((torch.abs(loc[o] - glob[o]).max() / torch.abs(glob[o]).max()).item() for o in ops3)
        eta_sweep[f"{eta:g}"] = {"ms": ms, "max_rel_diff_vs_global": diff}
    clk = clocks.stop()
    qbx.qbx_sync_status(plan)
    pairs = wl.n_ctr * wl.n_src
    per_op_terms = pairs * (2 * wl.p + 1)
    nops = {"S+D+grad S": 3, "R": 1, "grad D (PV)": 1, "S+D+grad S, r = 0.08 sqrt(h)": 3,
            "S+D+grad S, near-only eta = 8": 3, "S+D+grad S, 32 rhs": 3 * 32,
            "S, D, grad S via stored coefficients (form + eval)": 3, "S+D+grad S, k = 20 + 1i": 3,
            "S+D+grad S, 32 rhs, near-only eta = 8": 3 * 32, "S+D+grad S, 32 rhs, k = 20 + 1i": 3 * 32}
    print(json.dumps({
        "variants": f"starfish r=1+0.25cos5t, {wl.M} panels ({wl.n_tgt} targets, {wl.n_src} sources, "
                    f"{wl.n_ctr} centres), k=20, p=12, one CN(0,1) density (seed 2)",
        "steps": args.steps, "warmup": args.warmup,
        "l2": "flushed before every timed call (256 MiB write outside the event pair)",
        "ms": t,
        "terms_per_s": {name: nops[name] * per_op_terms / (ms * 1e-3) for name, ms in t.items()},
        "near_only_eta_sweep": eta_sweep,
        "clocks": clk}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-sample", type=int, default=1536, help="targets in the CPU-baseline sample (about 15 s of oracle work)")
    ap.add_argument("--ref-sample", type=int, default=48, help="targets per step of --impl reference")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched vs per-curve comparison (64 random curves)")
    ap.add_argument("--separate", action="store_true",
                    help="one qbx_apply launch per operator instead of one pass for all")
    ap.add_argument("--panels", type=int, default=None,
                    help="profiling only: override the panel count (smaller case for ncu)")
    ap.add_argument("--ops", default=None, help="profiling only: comma list of S,D,GRAD_S")
    ap.add_argument("--k", default=None, help="profiling only: override the wavenumber (complex: e.g. 20+1j)")
    ap.add_argument("--min-waves", type=int, default=None,
                    help="profiling only: qbx_plan_set_min_waves for the main step")
    ap.add_argument("--batch-steps", type=int, default=10, help="timed steps per arm of the batched comparison (>= 10)")
    ap.add_argument("--batch-curves", type=int, default=None,
                    help="profiling only: the first N curves of the batch")
    ap.add_argument("--batch-small", action="store_true",
                    help="with --batch-only: 256 small curves (16..48 panels) instead of the 64-curve workload")
    ap.add_argument("--batch-only", action="store_true",
                    help="profiling only: run the batched comparison alone and print it")
    ap.add_argument("--solve", action="store_true",
                    help="run the exterior scattering solve (1024-panel teardrop, 64 plane waves) instead")
    ap.add_argument("--variants", action="store_true",
                    help="time the R, grad D, r = c sqrt(h) and near-only variants on the full-size workload "
                         "instead")
    ap.add_argument("--adjoint", action="store_true",
                    help="time the forward, density-adjoint and shape-adjoint sweeps of the shape-optimisation "
                         "workload (128-panel starfish) instead")
    ap.add_argument("--solve-base", type=int, default=1008,
                    help="panels equispaced in t before the 2 x 8 corner bisections (profiling: smaller)")
    ap.add_argument("--assemble-only", action="store_true",
                    help="profiling only: with --solve, time the matrix assembly alone")
    ap.add_argument("--corner90", action="store_true",
                    help="with --solve: the teardrop with a 90-degree corner and the admissible radius rule")
    ap.add_argument("--matmul", action="store_true", help="the assembled solve's matrix product alone")
    ap.add_argument("--matmul-n", type=int, default=16384)
    ap.add_argument("--solve-matvec-only", action="store_true", help="profiling only: with --solve, time one matvec")
    ap.add_argument("--solve-restart", type=int, default=60)
    ap.add_argument("--solve-maxiter", type=int, default=400)
    args = ap.parse_args()
    if args.matmul:
        return run_matmul(args)
    if args.solve:
        return run_solve(args)
    if args.adjoint:
        return run_adjoint(args)
    if args.variants:
        return run_variants(args)
    if args.batch_only:
        import torch
        import paper_1207_4461_gb300 as qbx
        torch.cuda.set_device(0)
        print(json.dumps({"batched": run_batch_compare(args, qbx, torch)}))
        return 0
    wl = W.cfg2()
    if args.panels:
        wl.M = args.panels
    if args.ops:
        wl.ops = tuple(args.ops.split(","))
    if args.k:
        wl.k = complex(args.k) if "j" in args.k else float(args.k)
    if args.impl == "reference":
        return run_reference(args, wl)
    return run_gpu(args, wl)


if __name__ == "__main__":
    sys.exit(main())
