#!/usr/bin/env python
"""YAND-MVSK throughput on GB300: solves/s to kkt_rel <= 1e-8 at n=5440, T=12000.

One step = one batched frontier sweep: B = 64 instances (16 return targets x 4
preference vectors (1, 1, l3, l4), l3, l4 in {0.5, 2}) on one synthetic
fat-tailed GARCH factor panel, every instance solved from x0 = 1/n with its
mean coefficient calibrated to its target, through the library's C ABI.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun each rank solves its own copy
of the batch (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("solves/sec to rel ‖∇f‖≤1e-8 at n=5440,T=12000 "
          "(batched mixed vs plain FP64); HBM GB/s")
WORKLOAD = "c4_batch_n5440_T12000"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)  # ~0.7 s timed at C4: several clock samples
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["bf16", "fp32", "fp64"])
    ap.add_argument("--batch", type=int, default=64, help="instances per step (<= 64)")
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--lanes", type=int, default=0,
                    help="concurrent instances of the batched solver (0: all requests at once)")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 single-instance leg")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline leg")
    ap.add_argument("--max-elapsed", type=float, default=0.0,
                    help="per-request time limit in seconds (0: the library's); a profiler slows every launch")
    ap.add_argument("--sweep-panel", default="c4", choices=["c4", "c3"],
                    help="panel of the batched sweep: c4 (n=5440, T=12000; the measured workload) or c3 "
                         "(n=2000, T=12000: the same kernels on a smaller panel, for profiler captures)")
    ap.add_argument("--workload", default="c4",
                    choices=["c4", "paper-synthetic", "paper-line-search", "paper-conditioning", "warm-start"],
                    help="c4: the batched C4 sweep (default); paper-*: the paper's own benchmarks "
                         "(T=252 synthetic grid, exact vs Armijo step rule, CRRA conditioning sweep); "
                         "warm-start: the learned warm start (C5 panel), cold vs warm held-out solves")
    return ap.parse_args()


def dist_init(n):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("gloo")
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sweep_requests(world=1, panel="c4"):
    """The frontier sweep's requests: 4 preference vectors x 16 N return targets
    at asset-mean quantiles evenly spaced in [0.40, 0.85] (N = world size; the
    measured workload is N = 1: 64 requests, request q = 16 v + t).  More ranks
    add distinct targets, so every rank solves requests of its own.  panel
    "c3" puts the same requests on the n = 2000, T = 12000 GARCH panel."""
    import numpy as np

    import panels
    R, lams, _ = panels.workload(WORKLOAD)
    if panel == "c3":
        R, _, _ = panels.workload("c3_pcg_n2000_T12000")
    tg = panels.quantile_targets(R, np.linspace(0.40, 0.85, 16 * world))
    lam_b = np.asarray([l for l in lams for _ in tg])
    tg_b = np.asarray([t for _ in lams for t in tg])
    return R, lam_b, tg_b


def partition(n_requests, rank, world):
    """Indices of the global requests that rank `rank` solves: rank r takes
    r, r + N, r + 2N, ... (every request exactly once over the ranks)."""
    return list(range(rank, n_requests, world))


def gather_weights(W_local, idx_local, n_requests, world):
    """The weights of every request on rank 0, in global request order (W_local:
    rows of this rank's requests idx_local; host float64 array).  Other ranks
    receive None.  One gather over the process group (gloo for host tensors)."""
    import numpy as np
    if world == 1:
        out = np.empty((n_requests, W_local.shape[1]))
        out[idx_local] = W_local
        return out
    import torch
    import torch.distributed as dist
    obj = (list(idx_local), np.ascontiguousarray(W_local))
    parts = [None] * world if dist.get_rank() == 0 else None
    dist.gather_object(obj, parts, dst=0)
    if dist.get_rank() != 0:
        return None
    out = np.full((n_requests, W_local.shape[1]), np.nan)
    for idx, W in parts:
        out[idx] = W
    return out


def instances(batch, rank=0, world=1, panel="c4"):
    """This rank's share of the sweep (at most `batch` requests)."""
    R, lam_b, tg_b = sweep_requests(world, panel)
    idx = partition(len(lam_b), rank, world)[:batch]
    return R, lam_b[idx], tg_b[idx], idx


class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        self.f = None

    def start(self):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait(timeout=10)
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# The timed step brackets every PROF_STRIDE-th captured launch of its timed
# kinds with CUDA events (the average duration behind roofline.achieved).  A
# launch inside a replayed CUDA graph is bracketed on every replay when it is
# bracketed at capture, so the sampled count is not launches / PROF_STRIDE.
PROF_STRIDE = 5


def measured_traffic(kind):
    """DRAM bytes per launch of `kind` from profiles/traffic.json (an ncu
    capture), or None when absent or when its kernel sources changed since."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[kind]
        for path, digest in rec["sources"].items():
            if hashlib.sha256(open(os.path.join(ROOT, path), "rb").read()).hexdigest() != digest:
                return None
        return rec["bytes_per_launch"]
    except (OSError, ValueError, KeyError):
        return None


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# Secondary rooflines, from the fully profiled last warm-up step: the
# tensor-core products of the direction block (N = 576 fused / split, N = 64
# second PCG round) and the split FP64 products on the union.  The timed steps
# sample the dominant kind alone: it runs in the oracle block, so the
# direction bodies hold no profiler events and every iteration stays one
# graph (the library falls back to a host-selected body when they do).
SECONDARY_KINDS = ("gemm_tc_bf16_n192", "gemm_tc_bf16_n64", "oz_gemm_fwd_u")


def roofline_entry(name, d, pk, pk_src, T, n, ms_step, per_step=None):
    """Roofline of one profiled kind from its live CUDA-event durations.

    Tensor-core products report TFLOP/s against the sustained BF16 peak (the
    profiler's work figure is their FLOPs).  The N = 64 products and the split
    FP64 products are bandwidth-bound: they report GB/s of the operand they must
    stream once per launch (BF16 A: 2 T n bytes; the seven BF16 digit planes of
    the split product: 14 T n bytes, and the FP64 A it stands for, 8 T n)."""
    avg_s = d["total_ms"] / d["launches"] / 1e3
    # share: the average launch times the launches of one step (per_step, from
    # the fully profiled warm-up step), over the step's duration
    e = {"kernel": name, "sampled_launches": d["launches"], "launches_per_step": per_step,
         "avg_us": round(avg_s * 1e6, 2),
         "share_of_step": None if per_step is None else round(avg_s * 1e3 * per_step / ms_step, 4), "traffic": None}
    tr = measured_traffic(name)
    e["traffic"] = None if tr is None else round(tr)
    if name == "oz_gemm_fwd_u":
        # digit planes of the union's columns: 14 T |U| bytes; the profiler's
        # work is 56 T Bp |U| FLOPs (28 digit products, Bp = 64 vectors)
        byt = d["bytes_per_launch"] / (4.0 * 64)
        e.update({"bound": "hbm", "unit": "GB/s", "achieved": round(byt / avg_s / 1e9, 1), "peak": pk["hbm_gbs"],
                  "algorithmic_bytes": byt, "peak_source": pk_src})
    elif name.startswith("oz_gemm") and not name.endswith("_gated"):
        byt = 14.0 * T * n
        e.update({"bound": "hbm", "unit": "GB/s", "achieved": round(byt / avg_s / 1e9, 1), "peak": pk["hbm_gbs"],
                  "algorithmic_bytes": byt, "fp64_equivalent_gbs": round(8.0 * T * n / avg_s / 1e9, 1),
                  "peak_source": pk_src})
    elif name == "gemm_tc_bf16_n64":
        # the BF16 operand read once: FLOPs / N bytes (2 T K for K columns of A;
        # K = |U| on the face-restricted path, which the profiler counts per launch)
        byt = d["bytes_per_launch"] / 64.0
        e.update({"bound": "hbm", "unit": "GB/s", "achieved": round(byt / avg_s / 1e9, 1), "peak": pk["hbm_gbs"],
                  "algorithmic_bytes": byt, "peak_source": pk_src})
    elif name.startswith("gemm_tc"):
        e.update({"bound": "tensor", "unit": "TFLOP/s", "achieved": round(d["bytes_per_launch"] / avg_s / 1e12, 2),
                  "peak": pk["bf16_tflops_sustained"], "algorithmic_flops": d["bytes_per_launch"],
                  "peak_source": pk_src + " (sustained bf16)"})
    else:
        e.update({"bound": "hbm", "unit": "GB/s", "achieved": round(d["bytes_per_launch"] / avg_s / 1e9, 1),
                  "peak": pk["hbm_gbs"], "algorithmic_bytes": d["bytes_per_launch"], "peak_source": pk_src})
    e["frac"] = round(e["achieved"] / e["peak"], 4)
    return e


def plain_fp64(R, lam_b, tg_b, tol, picks):
    """The denominator of the headline ratio: the plain single-instance FP64
    GPU path (mvsk_solve on an FP64 context: FP64 streaming passes, one request
    at a time) on a stated subset of the same requests, each timed in full."""
    import numpy as np
    import torch

    import paper_2604_25378_gb300 as m
    ctx = m.MVSK(torch.from_numpy(R).cuda(), "fp64")
    ctx.set_prefs(np.asarray(lam_b[picks[0]]), float(tg_b[picks[0]]))
    ctx.solve(m.PCG, tol)  # untimed: first-use set-up of the context
    rows, total = [], 0.0
    for q in picks:
        ctx.set_prefs(np.asarray(lam_b[q]), float(tg_b[q]))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, info = ctx.solve(m.PCG, tol)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        total += dt
        rows.append({"request": int(q), "seconds": round(dt, 3), "iters": info["iters"], "evals": info["evals"],
                     "status": info["status"]})
    ctx.close()
    return {"solves_per_s": len(picks) / total, "requests": rows,
            "what": "mvsk_solve, FP64 context (FP64 streaming passes and FP64 Krylov vectors), one calibrated "
                    "request at a time, same tolerance"}


def run_ours(args, rank, world):
    import numpy as np
    import torch

    import paper_2604_25378_gb300 as m

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    R, lam_b, tg_b, idx = instances(args.batch, rank, world, args.sweep_panel)
    B = len(lam_b)
    T, n = R.shape
    Rd = torch.from_numpy(R).cuda()
    ctx = m.MVSK(Rd, args.precision)
    out = torch.empty((B, n), dtype=torch.float64, device="cuda")

    ctx.set_option("batch_lanes", args.lanes)
    if args.max_elapsed > 0:
        ctx.set_option("max_elapsed", args.max_elapsed)

    def step():
        return ctx.solve_batch(lam_b, tg_b, m.PCG, args.tol, out=out)

    # Warm-up; the last warm-up step runs with every launch profiled (the
    # breakdown), and the timed steps profile only their main kernel kinds.
    for w in range(args.warmup):
        if w == args.warmup - 1:
            ctx.profile_only(None)
            ctx.profile_enable(True)
        _, infos = step()
    torch.cuda.synchronize()
    breakdown, _ = ctx.profile_read()
    ctx.profile_enable(False)
    timed_kinds = {k: v for k, v in breakdown.items() if v["bytes_per_launch"] > 0 and not k.endswith("_gated")}
    dom_name = max(timed_kinds.items(), key=lambda kv: kv[1]["total_ms"])[0] if timed_kinds else None
    sampler = ClockSampler(torch.cuda.current_device())
    ctx.profile_only(dom_name if dom_name else "oz_gemm_bwd")
    # every PROF_STRIDE-th launch of each kind (an odd stride alternates the
    # two products of a Krylov step): each event node costs the graph an overlap
    ctx.profile_stride(PROF_STRIDE)
    ctx.profile_enable(True)
    barrier(world)
    torch.cuda.synchronize()
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    iters, lock = [], []
    torch.cuda.nvtx.range_push("timed_step")  # lets ncu restrict a capture to the timed region
    for _ in range(args.steps):
        _, infos = step()
        iters.append(sum(i["iters"] for i in infos))
        lock.append(infos[0]["batch_iters"])
    torch.cuda.nvtx.range_pop()
    e1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    barrier(world)
    ms = e0.elapsed_time(e1)
    prof, launches = ctx.profile_read()
    ctx.profile_enable(False)
    ctx.profile_stride(1)
    ms_max = max_over_ranks(ms, world)
    value = B * args.steps * world / (ms_max / 1e3)
    bad = [i for i in infos if i["status"] != "ok" or i["kkt_rel"] > args.tol]

    # Rooflines from the live CUDA-event durations of the timed steps: the
    # dominant kind, and the bandwidth-bound products beside it.
    pk, pk_src = peaks()
    # lanes doing useful work: live instance-iterations / (lockstep iterations x lanes)
    live = statistics.mean(iters) / (statistics.mean(lock) * B) if lock and lock[0] else None
    roof, secondary = None, []
    for name, d in sorted(prof.items(), key=lambda kv: -kv[1]["total_ms"]):
        if d["launches"] == 0 or name.endswith("_gated"):  # gated launches may skip their work
            continue
        roof = roofline_entry(name, d, pk, pk_src, T, n, ms / args.steps,
                              breakdown[name]["launches"] if name in breakdown else None)
        if live is not None:
            roof["live_lane_fraction"] = round(live, 4)
            roof["frac_useful"] = round(roof["frac"] * live, 4)
        break
    bd_ms = sum(v["total_ms"] for v in breakdown.values())
    for name in SECONDARY_KINDS:
        d = breakdown.get(name)
        if d is None or d["launches"] == 0 or (roof is not None and name == roof["kernel"]):
            continue
        e = roofline_entry(name, d, pk, pk_src, T, n, bd_ms, d["launches"])
        e["measured_in"] = "last warm-up step (every launch profiled; share of its summed kernel time)"
        secondary.append(e)

    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16+f64" if args.precision == "bf16" else
            ("fp32+f64" if args.precision == "fp32" else "f64"), "data": "synthetic",
            "config": {"workload": WORKLOAD if args.sweep_panel == "c4" else "c3_panel_batch_n2000_T12000",
                       "n": n, "T": T, "instances_per_gpu": B,
                       "targets": 16, "preference_vectors": 4, "configuration": "pcg",
                       "tol": args.tol, "start": "1/n (cold)",
                       "l2": "inputs larger than L2: A is 522 MB FP64 + 131 MB BF16",
                       "parallelism": f"request partition x{world}" if world > 1 else "single device"},
            "precision": args.precision,
            "gpu_launches": int(launches), "roofline": roof, "roofline_secondary": secondary, "clocks": clocks,
            "solve_iterations_per_step": statistics.mean(iters) if iters else None,
            "lockstep_iterations_per_step": statistics.mean(lock) if lock else None,
            "request_iterations": {"min": min(i["iters"] for i in infos), "max": max(i["iters"] for i in infos),
                                   "mean": statistics.mean(i["iters"] for i in infos)},
            "request_inner_solves": {"min": min(i["evals"] for i in infos), "max": max(i["evals"] for i in infos),
                                     "mean": statistics.mean(i["evals"] for i in infos)},
            "unconverged_instances": len(bad)}

    e2e = None
    if not args.no_e2e:
        # Same metric through the public API with host buffers: pinned R in,
        # weights out, every step (context creation = H2D copy + centring).
        Rh = torch.from_numpy(R).pin_memory()
        Wh = torch.empty((B, n), dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            c2 = m.MVSK(Rh, args.precision)
            c2.set_option("batch_lanes", args.lanes)
            c2.solve_batch(lam_b, tg_b, m.PCG, args.tol, out=Wh)
            c2.close()
        torch.cuda.synchronize()
        dt = max_over_ranks(time.perf_counter() - t0, world)
        e2e = {"value": B * args.steps * world / dt, "unit": "solves/s",
               "h2d_bytes_per_step": int(R.nbytes + lam_b.nbytes + tg_b.nbytes),
               "d2h_bytes_per_step": int(Wh.numel() * 8)}
        # every request's weights on rank 0, in global order (outside the timed region)
        Wall = gather_weights(Wh.numpy(), idx, B * world, world)
        if rank == 0:
            line["gathered_requests"] = int(np.sum(np.isfinite(Wall).all(axis=1)))
    line["e2e"] = e2e
    ctx.close()
    if rank == 0 and not args.no_plain:
        # the plain FP64 single-instance path on one request of each preference
        # vector (targets spread over the grid): the headline ratio's denominator
        picks = [0, 21, 42, 63][: max(1, min(4, B))]
        pf = plain_fp64(R, lam_b, tg_b, args.tol, picks)
        line["plain_fp64"] = pf
        line["speedup_vs_plain_fp64"] = round(value / world / pf["solves_per_s"], 2)
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(args, R, lam_b, tg_b)
    line["breakdown_last_warmup_step"] = {k: {"launches": v["launches"], "ms": round(v["total_ms"], 3)}
                                          for k, v in sorted(breakdown.items(), key=lambda kv: -kv[1]["total_ms"])}
    return line


def blas_threads():
    """Threads the host BLAS uses (the oracle's only parallel part)."""
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        v = os.environ.get(k)
        if v and v.isdigit():
            return int(v)
    return os.cpu_count()


def oracle_request_solve(A, mu, lam, target, tol):
    """One complete calibrated request as the oracle, as it stands, solves it:
    standardised coefficients, c1 calibrated to the target (Sec. 6), every
    inner solve Alg. 1 in the PCG configuration.  Returns (seconds, YAND
    iterations summed over the inner solves, inner solves)."""
    from oracle import mvsk_oracle as O
    its = [0]

    def count(it, x, rel):
        its[0] += 1

    c = O.scale_preferences(lam, A, "standardised")
    t0 = time.perf_counter()
    _, _, _, ev = O.calibrate_target(A, mu, c, target, "pcg", tol, opts=None, callback=count)
    return time.perf_counter() - t0, its[0], ev


# Requests of the sweep visited by the CPU legs, in this order: q = 17 i mod
# 64 walks the four preference vectors and the targets together.
def cpu_request_order(k, nreq=64):
    return [(17 * i) % nreq for i in range(k)]


def cpu_baseline(args, R, lam_b, tg_b):
    """The oracle, as it stands, on the host cores: complete calibrated solves
    of a bounded sample of the sweep's requests (CPU_REQUESTS of them)."""
    from oracle import mvsk_oracle as O
    mu, A = O.centre(R)
    qs = cpu_request_order(CPU_REQUESTS, len(lam_b))
    secs, its = 0.0, 0
    for q in qs:
        dt, it, _ = oracle_request_solve(A, mu, lam_b[q], tg_b[q], args.tol)
        secs += dt
        its += it
    return {"value": len(qs) / secs, "unit": "solves/s", "cores": blas_threads(), "kind": "oracle",
            "sample": f"complete calibrated oracle solves of requests {qs} of the sweep (numpy FP64, "
                      f"{blas_threads()} BLAS threads): {secs:.1f} s, {its} YAND iterations"}


CPU_REQUESTS = 2


def run_reference(args, rank, world):
    """The oracle as the reference arm: each step is one complete calibrated
    solve of one request of the sweep (requests in cpu_request_order), timed
    with the wall clock; W untimed steps first."""
    if rank != 0:
        return None
    from oracle import mvsk_oracle as O
    R, lam_b, tg_b, _ = instances(args.batch)
    mu, A = O.centre(R)
    order = cpu_request_order(args.warmup + args.steps, len(lam_b))
    times, its = [], 0
    for k, q in enumerate(order):
        dt, it, _ = oracle_request_solve(A, mu, lam_b[q], tg_b[q], args.tol)
        if k >= args.warmup:
            times.append(dt)
            its += it
    secs = sum(times)
    v = len(times) / secs if secs > 0 else None
    timed = order[args.warmup:]
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(1, len(times)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": R.shape[1], "T": R.shape[0], "instances_per_gpu": len(lam_b),
                       "targets": 16, "preference_vectors": 4, "configuration": "pcg",
                       "tol": args.tol, "start": "1/n (cold)",
                       "l2": "inputs larger than L2: A is 522 MB FP64 + 131 MB BF16",
                       "parallelism": "single device"},
            "precision": "fp64 (CPU oracle)",
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": blas_threads(), "kind": "oracle",
                             "sample": f"one complete calibrated oracle solve per step, requests {timed} "
                                       f"({its} YAND iterations in {secs:.1f} s)"},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "note": "the CPU oracle (numpy FP64) as it stands: there is no other reference implementation"}


# The paper's published YAND-MVSK means on its synthetic benchmark (Table
# synthetic-summary; hardware not stated): seconds, iterations, projected residual.
PAPER_SYNTHETIC_YAND = {"small": {"mean_time_s": 0.0711, "mean_iters": 41.74, "mean_residual": 2.69e-7, "runs": 54},
                        "large": {"mean_time_s": 0.332, "mean_iters": 98.56, "mean_residual": 3.56e-6, "runs": 48}}


def run_paper_synthetic(args, rank, world):
    """The paper's synthetic benchmark grid, one single-instance FP64 solve per
    (dimension, profile) from 1/n: direct for n <= 100, PCG beyond.  Times are
    wall-clock per mvsk_solve call (context and profile set up outside)."""
    if rank != 0:
        return None
    import numpy as np
    import torch

    import panels
    import paper_2604_25378_gb300 as m
    g = panels.PAPER_SYNTHETIC
    runs = []
    for regime, ns, cfg in (("small", g["small_n"], m.DIRECT), ("large", g["large_n"], m.PCG)):
        for n in ns:
            R = panels.uniform_panel(n, g["T"], n)
            ctx = m.MVSK(torch.from_numpy(R).cuda(), "fp64")
            ctx.set_option("pref_scaling", 0)
            for prof in g["profiles"]:
                ctx.set_prefs(np.asarray(prof, dtype=np.float64))
                for _ in range(max(args.warmup, 0)):
                    ctx.solve(cfg, args.tol)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                _, info = ctx.solve(cfg, args.tol)
                dt = time.perf_counter() - t0
                runs.append({"regime": regime, "n": n, "profile": list(prof), "seconds": dt, "iters": info["iters"],
                             "kkt": info["kkt_residual"], "status": info["status"]})
            ctx.close()

    def summary(rs):
        return {"runs": len(rs), "mean_time_s": statistics.mean(r["seconds"] for r in rs),
                "mean_iters": statistics.mean(r["iters"] for r in rs),
                "mean_residual": statistics.mean(r["kkt"] for r in rs),
                "converged": sum(r["status"] == "ok" for r in rs)}

    small = summary([r for r in runs if r["regime"] == "small"])
    large = summary([r for r in runs if r["regime"] == "large"])
    return {"metric": "mean seconds per solve, paper synthetic benchmark (T=252, n=4..5000)",
            "value": statistics.mean(r["seconds"] for r in runs), "unit": "s", "n_gpus": 1,
            "higher_is_better": False, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "paper_synthetic_T252", "T": g["T"], "small_n": g["small_n"],
                       "large_n": g["large_n"], "profiles": g["profiles"], "tol": args.tol,
                       "configuration": "direct for n <= 100, pcg beyond", "warmup_solves_per_run": args.warmup},
            "small": small, "large": large, "paper_reported": PAPER_SYNTHETIC_YAND,
            "per_dimension": [{k: r[k] for k in ("regime", "n", "seconds", "iters", "kkt", "status")} for r in runs]}


# Table yand-line-search (direct configuration, n in {4, 8, 12}, T = 252).
PAPER_LINE_SEARCH = {"armijo": {"mean_time_s": 1.40e-2, "median_time_s": 9.93e-3, "mean_iters": 29.8,
                                "mean_residual": 3.61e-7},
                     "exact": {"mean_time_s": 1.17e-2, "median_time_s": 4.18e-3, "mean_iters": 19.0,
                               "mean_residual": 8.21e-8}}
# Tables crra-conditioning (n = 1000, T = 2000) and crra-conditioning-stress
# (n = 5000, T = 252): median seconds and median projected residual of YAND (large).
PAPER_CONDITIONING = {"n1000_T2000": {"1": (0.122, 1.28e-6), "10": (0.399, 1.27e-6), "100": (0.482, 1.36e-6),
                                      "1000": (0.423, 1.40e-6)},
                      "n5000_T252": {"1": (0.569, 5.02e-6), "10": (1.270, 5.37e-6), "100": (1.291, 5.99e-6),
                                     "1000": (1.394, 6.61e-6)}}


def _timed_solve(ctx, cfg, tol, warmup):
    import torch
    for _ in range(warmup):
        ctx.solve(cfg, tol)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, info = ctx.solve(cfg, tol)
    return time.perf_counter() - t0, info


def run_paper_line_search(args, rank, world):
    """Table yand-line-search: direct configuration, exact quartic vs Armijo
    backtracking, n in {4, 8, 12}, T = 252, the three raw profiles."""
    if rank != 0:
        return None
    import numpy as np
    import torch

    import panels
    import paper_2604_25378_gb300 as m
    out = {}
    for rule, code in (("exact", 0), ("armijo", 1)):
        rows = []
        for n in (4, 8, 12):
            R = panels.uniform_panel(n, 252, n)
            ctx = m.MVSK(torch.from_numpy(R).cuda(), "fp64")
            ctx.set_option("pref_scaling", 0)
            ctx.set_option("line_search", code)
            if code == 1:
                ctx.set_option("max_iter", 120)  # Table yand-core-parameters, Armijo diagnostic row
            for prof in panels.PAPER_SYNTHETIC["profiles"]:
                ctx.set_prefs(np.asarray(prof))
                dt, info = _timed_solve(ctx, m.DIRECT, args.tol, max(args.warmup, 0))
                rows.append((dt, info["iters"], info["kkt_residual"], info["status"] == "ok"))
            ctx.close()
        out[rule] = {"runs": len(rows), "mean_time_s": statistics.mean(r[0] for r in rows),
                     "median_time_s": statistics.median(r[0] for r in rows),
                     "mean_iters": statistics.mean(r[1] for r in rows),
                     "mean_residual": statistics.mean(r[2] for r in rows), "converged": sum(r[3] for r in rows)}
    return {"metric": "mean seconds per solve, direct configuration, exact vs Armijo step (T=252, n=4,8,12)",
            "value": out["exact"]["mean_time_s"], "unit": "s", "n_gpus": 1, "higher_is_better": False,
            "dtype": "f64", "data": "synthetic", "config": {"workload": "paper_line_search_T252", "tol": args.tol},
            "exact": out["exact"], "armijo": out["armijo"], "paper_reported": PAPER_LINE_SEARCH}


def run_paper_conditioning(args, rank, world):
    """Tables crra-conditioning / crra-conditioning-stress: gamma = 6 CRRA
    coefficients, prescribed kappa_+(A U), PCG configuration with stall
    recovery, three instances per level, one untimed warm-up solve each; medians."""
    if rank != 0:
        return None
    import numpy as np
    import torch

    import panels
    import paper_2604_25378_gb300 as m
    out = {}
    for key, n, T in (("n1000_T2000", 1000, 2000), ("n5000_T252", 5000, 252)):
        out[key] = {}
        for kappa in (1.0, 10.0, 100.0, 1000.0):
            rows = []
            for seed in range(3):
                R = panels.crra_conditioning_panel(n, T, kappa, 100 + seed)
                ctx = m.MVSK(torch.from_numpy(R).cuda(), "fp64")
                ctx.set_option("pref_scaling", 0)
                ctx.set_prefs(np.asarray(panels.CRRA_GAMMA6))
                dt, info = _timed_solve(ctx, m.PCG, args.tol, max(args.warmup, 1))
                rows.append((dt, info["kkt_residual"], info["iters"], info["status"] == "ok"))
                ctx.close()
            out[key][str(int(kappa))] = {"median_time_s": statistics.median(r[0] for r in rows),
                                         "median_residual": statistics.median(r[1] for r in rows),
                                         "median_iters": statistics.median(r[2] for r in rows),
                                         "converged": sum(r[3] for r in rows)}
    return {"metric": "median seconds per solve, CRRA conditioning benchmark (gamma=6, PCG)",
            "value": statistics.median(v["median_time_s"] for v in out["n1000_T2000"].values()), "unit": "s",
            "n_gpus": 1, "higher_is_better": False, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "paper_crra_conditioning", "tol": args.tol, "instances_per_level": 3},
            "levels": out, "paper_reported_median_time_s_and_residual": PAPER_CONDITIONING}


def run_warm_start(args, rank, world):
    """The learned warm start on a C5-style panel (n = 5440, T = 12000, seed
    100): solver outputs of WS_TRAIN requests train the network (features of
    the request and the panel statistics -> n w*), then WS_TEST held-out
    requests are solved through 64 lanes (continuous batching) from 1/n and
    from the network's projected output; solves/s and mean YAND iterations of
    both (requests with a target start their calibration from 1/n either way)."""
    if rank != 0:
        return None
    import numpy as np
    import torch

    import panels
    import paper_2604_25378_gb300 as m
    n, T = 5440, 12000
    R = panels.garch_sector_panel(n, T, 100)
    ctx = m.MVSK(torch.from_numpy(R).cuda(), args.precision)
    mu, sg = ctx.column_stats()
    rng = np.random.default_rng(101)
    qs_all = np.quantile(R.mean(axis=0), np.linspace(0.40, 0.85, 64))

    def requests(k):
        lam = np.column_stack([np.ones(k), np.ones(k), rng.choice([0.5, 1.0, 2.0], k) * rng.uniform(0.8, 1.25, k),
                               rng.choice([0.5, 1.0, 2.0], k) * rng.uniform(0.8, 1.25, k)])
        tg = np.where(rng.uniform(size=k) < 0.5, np.nan, rng.choice(qs_all, k))
        return lam, tg

    ctx.set_option("batch_lanes", 64)  # requests queue for 64 lanes (continuous batching)

    def solve(lam, tg, W0=None):
        out = torch.empty((lam.shape[0], n), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        W, infos = ctx.solve_batch(lam, tg, m.PCG, args.tol, W0=W0, out=out)
        torch.cuda.synchronize()
        assert all(i["status"] == "ok" for i in infos), [i["status"] for i in infos]
        return W, [i["iters"] for i in infos], time.perf_counter() - t0

    lam_tr, tg_tr = requests(WS_TRAIN)
    Wtr, its_tr, t_data = solve(lam_tr, tg_tr)
    X_tr = m.MLP.features(mu, sg, lam_tr, tg_tr, WS_SEED)
    Y_tr = (Wtr * n).float().contiguous()
    net = m.MLP(d_in=m.MLP_D_IN, d_hidden=512, n_hidden=4, d_out=n, max_batch=WS_TEST, seed=WS_SEED)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = []
    for ep in range(WS_EPOCHS):
        perm = torch.randperm(WS_TRAIN, device="cuda")
        for k in range(WS_TRAIN // 128):
            idx = perm[k * 128:(k + 1) * 128]
            losses.append(net.train_step(X_tr[idx].contiguous(), Y_tr[idx].contiguous(),
                                         1e-3 if ep < WS_EPOCHS * 2 // 3 else 2e-4))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    lam_te, tg_te = requests(WS_TEST)
    solve(lam_te[:64], tg_te[:64])  # untimed warm-up
    Wc, its_c, t_cold = solve(lam_te, tg_te)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    X_te = m.MLP.features(mu, sg, lam_te, tg_te, WS_SEED)
    W0 = net.warm_start(X_te, n, 1e-8)
    torch.cuda.synchronize()
    t_infer = time.perf_counter() - t0
    Ww, its_w, t_warm = solve(lam_te, tg_te, W0)
    dev = float((Ww - Wc).abs().max())
    return {"metric": "solves/s of held-out requests with the learned warm start (C5 panel, 64 lanes)",
            "value": WS_TEST / (t_warm + t_infer), "unit": "solves/s", "n_gpus": 1, "higher_is_better": True,
            "dtype": "bf16+f64", "data": "synthetic",
            "config": {"workload": "c5_warm_start_n5440_T12000", "n": n, "T": T, "panel_seed": 100,
                       "train_requests": WS_TRAIN, "test_requests": WS_TEST, "epochs": WS_EPOCHS,
                       "network": "128 -> 4 x 512 ReLU -> 5440, BF16 tcgen05 GEMMs, Adam", "tol": args.tol},
            "cold": {"solves_per_s": WS_TEST / t_cold, "mean_iters": float(np.mean(its_c))},
            "warm": {"solves_per_s": WS_TEST / (t_warm + t_infer), "mean_iters": float(np.mean(its_w)),
                     "inference_s": t_infer},
            "train": {"data_solve_s": t_data, "train_s": t_train, "first_loss": losses[0], "last_loss": losses[-1],
                      "mean_iters_of_data": float(np.mean(its_tr))},
            "max_abs_w_difference_warm_vs_cold": dev}


# Learned warm start workload: requests solved for training data, held out, epochs.
WS_TRAIN, WS_TEST, WS_EPOCHS, WS_SEED = 768, 256, 200, 31


def main():
    args = parse()
    rank, world = dist_init(args.gpus)
    if args.impl == "reference":
        line = run_reference(args, rank, world)
    elif args.workload == "paper-synthetic":
        line = run_paper_synthetic(args, rank, world)
    elif args.workload == "paper-line-search":
        line = run_paper_line_search(args, rank, world)
    elif args.workload == "paper-conditioning":
        line = run_paper_conditioning(args, rank, world)
    elif args.workload == "warm-start":
        line = run_warm_start(args, rank, world)
    else:
        line = run_ours(args, rank, world)
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
