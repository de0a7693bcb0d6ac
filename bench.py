#!/usr/bin/env python
"""Benchmark of the sketching hot path on the tall regression workload.

Workload (seeded, synthetic): A is 1,048,576 x 256 FP32 with N(0,1) entries times a per-row lognormal(0,1)
factor, b = A x* + N(0, 1e-3) noise.  One step = one sketch-and-solve (rmc_lsr_sketch: [A, b] sketched in
one pass, then the FP64 solve) for each sketch kind (count sketch, SRHT, Gaussian) and each sketch size
s in {1024, 4096}: six calls.  The metric is sketch throughput in GB/s: the algorithmic bytes of the six
calls (read A and b, write the s x 257 sketch) divided by the step time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun, one process per GPU): every rank runs its own replica of the workload (the path has no
data exchange); value = bytes of all ranks / max over ranks of the timed region ("scaling": "weak").
--impl reference times the FP64 CPU oracle on the host cores on a bounded sample of the same workload.
"""
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

M, N_COLS = 1 << 20, 256
STEP = [("countsketch", 1024), ("countsketch", 4096), ("srht", 1024), ("srht", 4096),
        ("gaussian", 1024), ("gaussian", 4096)]
SEED = 20150527
ORACLE_SAMPLE_ROWS = 4096          # rows of A the CPU oracle sketches per call
GAUSS_PREC = os.environ.get("RMC_BENCH_GAUSS_PREC", "tf32")
# DRAM bytes per row of A per launch from ncu captures of `python bench.py --probe <kind>` (A 262,144 x 256 + b):
# dram__bytes_read.sum + dram__bytes_write.sum divided by 262,144.  Re-capture when a kernel changes.
PROFILED_DRAM_BYTES_PER_ROW = {
    "gaussian_sketch": (271.001344e6 + 5.668096e6) / 262144,
    "srht_stage1": (268.572928e6 + 42.968832e6) / 262144,
    "countsketch_gather": (271.636992e6 + 3.304704e6) / 262144,
}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return {"hbm_gbs": p["hbm_gbs"], "bf16_tflops": p["bf16_tflops"], "sm_max_mhz": p.get("sm_max_mhz", 2070.0),
                "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0, "source": "fallback"}


def call_bytes(m, n, s):
    """Algorithmic bytes of one sketch of [A, b]: read A and b once, write the s x (n+1) sketch."""
    return 4 * (m * n + m + s * (n + 1))


# ------------------------------------------------------------------------------------------ rank helpers

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def combine_over_ranks(seconds, nbytes, world):
    """(max time over ranks, total bytes over ranks); identity at world size 1."""
    if world == 1:
        return seconds, nbytes
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([seconds], dtype=torch.float64, device=dev)
    b = torch.tensor([float(nbytes)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(b, op=dist.ReduceOp.SUM)
    return float(t.item()), float(b.item())


# ------------------------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.rows = []
        if self.proc is None:
            return False
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)
        return False

    def summary(self):
        if not getattr(self, "rows", None):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ------------------------------------------------------------------------------------------- CPU arm

def oracle_sample(seconds_budget=None):
    """The FP64 oracle as it stands, on the first ORACLE_SAMPLE_ROWS rows of the workload recipe (drawn on the
    CPU), for every call of the step.  Returns (GB/s, seconds, bytes, description)."""
    import numpy as np
    import workloads
    from oracle import lsr
    A, b, _ = workloads.tall_lsr_numpy(ORACLE_SAMPLE_ROWS, N_COLS, seed=SEED)
    nbytes = 0
    t0 = time.perf_counter()
    for kind, s in STEP:
        s_eff = min(s, ORACLE_SAMPLE_ROWS)
        lsr.lsr_sketch(A, b, s_eff, kind, SEED)
        nbytes += call_bytes(ORACLE_SAMPLE_ROWS, N_COLS, s_eff)
    dt = time.perf_counter() - t0
    desc = ("oracle lsr_sketch (FP64 NumPy) for the 6 calls of one step on a %d x %d sample of the workload "
            "(s capped at the sample's rows); GB/s = algorithmic bytes of the sample / wall time" %
            (ORACLE_SAMPLE_ROWS, N_COLS))
    return nbytes / dt / 1e9, dt, nbytes, desc


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    cores = os.cpu_count()
    for _ in range(args.warmup):
        oracle_sample()
    total_b, total_t = 0, 0.0
    for _ in range(args.steps):
        _, dt, nb, desc = oracle_sample()
        total_b += nb
        total_t += dt
    value = total_b / total_t / 1e9
    line = {
        "impl": "reference", "metric": "sketch HBM GB/s", "value": value, "unit": "GB/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total_t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "tall-lsr sample %dx%d (6 sketch-and-solve calls per step)" % (ORACLE_SAMPLE_ROWS, N_COLS)},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------------------------------- GPU arm

def union_ms(spans):
    """Length of the union of [start, stop) intervals (milliseconds)."""
    total, end = 0.0, None
    for a, b in sorted(spans):
        if end is None or a > end:
            total += b - a
            end = b
        elif b > end:
            total += b - end
            end = b
    return total


def run_ours(args, world, rank, local):
    import torch
    import paper_1505_07570_gb300 as rmc
    import workloads

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    A, b, _ = workloads.tall_lsr_torch(M, N_COLS, seed=SEED + rank)
    torch.cuda.synchronize()
    step_bytes = sum(call_bytes(M, N_COLS, s) for _, s in STEP)

    # the six calls are independent and each runs on its own stream, so every call's small solve kernels
    # overlap the other calls' sketches; the library keeps one context per stream
    streams = {(kind, s): torch.cuda.Stream() for kind, s in STEP}
    main = torch.cuda.current_stream()

    def step(outs=None, A_in=None, b_in=None):
        A_in = A if A_in is None else A_in
        b_in = b if b_in is None else b_in
        for kind, s in STEP:
            st = streams[(kind, s)]
            st.wait_stream(main)
            with torch.cuda.stream(st):
                x = rmc.rmc_lsr_sketch(A_in, b_in, s, kind, SEED, prec=GAUSS_PREC if kind == "gaussian" else "fp32")
            if outs is not None:
                outs.append(x)
        for st in streams.values():
            main.wait_stream(st)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        step()
    rmc.rmc_sync_all()
    stream = torch.cuda.current_stream()
    launches0 = rmc.rmc_launch_counter()
    rmc.rmc_profile_begin()
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        rmc.rmc_profile_reference()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
    rmc.rmc_sync_all()
    seconds = ev0.elapsed_time(ev1) / 1e3
    launches = rmc.rmc_launch_counter() - launches0
    kernels = {}
    for name, tag in [("countsketch_gather", rmc.K_COUNTSKETCH), ("srht_stage1", rmc.K_SRHT),
                      ("srht_stage2", rmc.K_SRHT_REDUCE), ("gaussian_sketch", rmc.K_GAUSSIAN),
                      ("gram_fp64", rmc.K_GRAM), ("small_fp64", rmc.K_SMALL)]:
        cnt, ms = rmc.rmc_profile_read(tag)
        if cnt:
            kernels[name] = {"launches": cnt, "ms_total": ms, "ms_busy": union_ms(rmc.rmc_profile_spans(tag))}
    rmc.rmc_profile_end()
    tmax, total_bytes = combine_over_ranks(seconds, step_bytes * args.steps, world)

    # e2e: inputs copied from pinned host memory every step, results read back
    A_h = A.cpu().pin_memory()
    b_h = b.cpu().pin_memory()
    h2d = A_h.numel() * 4 + b_h.numel() * 4
    # Two device copies of the inputs: step k+1's host-to-device copy runs on its own stream while step k
    # computes on the other buffer (each step still copies all of its inputs and reads its result back).
    bufs = [(A, b), (torch.empty_like(A), torch.empty_like(b))]
    copy_stream = torch.cuda.Stream()
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    used = [torch.cuda.Event(), torch.cuda.Event()]

    def copy_in(k):
        Ab, bb_ = bufs[k % 2]
        copy_stream.wait_event(used[k % 2])  # the step that last read this buffer is done
        with torch.cuda.stream(copy_stream):
            Ab.copy_(A_h, non_blocking=True)
            bb_.copy_(b_h, non_blocking=True)
            copied[k % 2].record(copy_stream)

    def e2e_steps(n):
        host = []
        for u in used:
            u.record(stream)
        copy_in(0)
        for k in range(n):
            if k + 1 < n:
                copy_in(k + 1)
            stream.wait_event(copied[k % 2])
            outs = []
            step(outs, *bufs[k % 2])
            used[k % 2].record(stream)
            host = [x.to("cpu", non_blocking=False) for x in outs]
        return host

    e2e_steps(max(1, args.warmup))
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    xs = e2e_steps(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    d2h = sum(x.numel() * 8 for x in xs)
    e2e_seconds, _ = combine_over_ranks(e0.elapsed_time(e1) / 1e3, 0, world)
    e2e_value = step_bytes * args.steps * world / e2e_seconds / 1e9
    assert all(bool(torch.isfinite(x).all()) for x in xs)
    # the host-to-device copy alone (pinned host memory, the copy stream, nothing else running): the e2e step
    # cannot beat max(device step, this copy)
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(copy_stream):
        c0.record(copy_stream)
        for _ in range(3):
            bufs[1][0].copy_(A_h, non_blocking=True)
            bufs[1][1].copy_(b_h, non_blocking=True)
        c1.record(copy_stream)
    torch.cuda.synchronize()
    h2d_ms = c0.elapsed_time(c1) / 3

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return 0

    pk = peaks()
    value = total_bytes / tmax / 1e9

    def roofline_of(name, rec):
        """Roofline entry of one sketch kernel from its launch count and device time: the union of its launches'
        event intervals where launches of the kernel overlap (in the step the calls run on their own streams, and
        a launch's event pair also spans its wait for another launch's CTAs), else the summed event time."""
        avg_s = rec.get("ms_busy", rec["ms_total"]) / rec["launches"] / 1e3
        kind = name.split("_")[0]
        if kind == "gaussian":
            # per launch: one (kind, s) call; flops of the product, averaged over the two sketch sizes
            flops = sum(2.0 * M * s * (N_COLS + 1) for k, s in STEP if k == "gaussian") / 2
            if GAUSS_PREC == "fp32":
                peak = 152 * 128 * 2 * pk["sm_max_mhz"] * 1e6 / 1e12
                r = {"bound": "alu", "achieved": flops / avg_s / 1e12, "peak": peak, "unit": "TFLOP/s",
                     "peak_source": "152 SMs x 128 FP32 FMA/clk x 2 x max SM clock"}
            else:
                ratio = 1.1 / 2.25 if GAUSS_PREC == "tf32" else 1.0
                r = {"bound": "tensor", "achieved": flops / avg_s / 1e12, "peak": pk["bf16_tflops"] * ratio,
                     "unit": "TFLOP/s", "peak_source": "%s bf16 x nominal %s/bf16 ratio" % (pk["source"], GAUSS_PREC)}
        else:
            per_launch = sum(call_bytes(M, N_COLS, s) for k, s in STEP if k == kind) / 2
            r = {"bound": "hbm", "achieved": per_launch / avg_s / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s",
                 "peak_source": pk["source"]}
        r["frac"] = r["achieved"] / r["peak"]
        r["kernel"] = name
        r["timing"] = ("union of the launches' CUDA-event intervals in the timed region" if "ms_busy" in rec
                       else "summed CUDA-event time of the launches, one call at a time")
        r["ms_avg"] = avg_s * 1e3
        # dram__bytes_read.sum + dram__bytes_write.sum of one launch, captured on the 262,144-row probe and
        # scaled by rows to this workload (each kernel reads every row once, so traffic grows in proportion)
        per_row = PROFILED_DRAM_BYTES_PER_ROW.get(name)
        r["traffic"] = per_row * M if per_row else None
        return r

    sketch_kernels = {k: v for k, v in kernels.items() if k in ("countsketch_gather", "srht_stage1", "gaussian_sketch")}
    roof = None
    if sketch_kernels:
        name, rec = max(sketch_kernels.items(), key=lambda kv: kv[1]["ms_total"])
        roof = roofline_of(name, rec)
    for name, rec in kernels.items():
        rec["ms_avg"] = rec["ms_total"] / rec["launches"]
    # the same kernels once more, one call at a time on one stream (no overlap), for per-kernel rooflines
    isolated = {}
    rmc.rmc_profile_begin()
    for kind, s in STEP:
        with torch.cuda.stream(streams[(kind, s)]):
            rmc.rmc_lsr_sketch(A, b, s, kind, SEED, prec=GAUSS_PREC if kind == "gaussian" else "fp32")
        torch.cuda.synchronize()
    for name, tag in [("countsketch_gather", rmc.K_COUNTSKETCH), ("srht_stage1", rmc.K_SRHT),
                      ("gaussian_sketch", rmc.K_GAUSSIAN)]:
        cnt, ms = rmc.rmc_profile_read(tag)
        if cnt:
            isolated[name] = roofline_of(name, {"launches": cnt, "ms_total": ms})
    rmc.rmc_profile_end()

    forms_info = None
    if world == 1:
        forms_info = gaussian_forms_measure(torch, rmc, A, b)
    precise_info = None
    if world == 1 and not args.no_rsvd:
        precise_info = precise_measure(torch, rmc, A, b)
    rsvd_info = None
    if world == 1 and not args.no_rsvd:
        del A_h, b_h
        rsvd_info = rsvd_measure(torch, rmc)
    batch_info = None
    if world == 1 and not args.no_batch:
        batch_info = batch_measure(torch, rmc)
    serve_info = None
    if world == 1 and not args.no_serve:
        serve_info = serve_measure(torch, rmc, rates=tuple(int(r) for r in args.serve_rates.split(",")),
                                   window_s=args.serve_window, nstreams=args.serve_streams)

    cpu = None
    if world == 1:
        v, dt, nb, desc = oracle_sample()
        cpu = {"value": v, "unit": "GB/s", "cores": os.cpu_count(), "kind": "oracle", "sample": desc}

    line = {
        "metric": "sketch HBM GB/s", "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * tmax / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "tall-lsr 1048576x256 FP32 + b; step = lsr_sketch x {countsketch, srht, gaussian}"
                               " x s {1024, 4096}", "gaussian_prec": GAUSS_PREC, "l2": "inputs (1.07 GB) > L2",
                   "parallelism": "replicas" if world > 1 else "single"},
        "roofline": roof, "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "GB/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": 1e3 * e2e_seconds / args.steps, "h2d_alone_ms": h2d_ms,
                "h2d_alone_gbs": h2d / h2d_ms / 1e6},
        "gpu_launches": launches, "clocks": clk.summary(), "kernels": kernels, "kernels_isolated": isolated,
        "gaussian_forms": forms_info, "lsr_precise": precise_info, "rsvd": rsvd_info, "batch": batch_info,
        "serve": serve_info,
    }
    print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_probe(kind):
    """One small case of one kernel family, for profiler captures: A 262,144 x 256 (+ b), two warm-up calls,
    then two timed calls.  Prints one JSON line."""
    import torch
    import paper_1505_07570_gb300 as rmc
    import workloads
    if kind == "peaks":
        return matmul_peaks(torch)
    if kind == "batch":
        info = batch_measure(torch, rmc, count=512, m_range=(512, 8192), reps=2)
        print(json.dumps({"probe": kind, "ms_per_call": info["ms"], "info": info}))
        return 0
    A, b, _ = workloads.tall_lsr_torch(1 << 18, N_COLS, seed=SEED)
    if kind == "rsvd":
        A = workloads.factor_rank_torch(16384, 4096, 512, seed=SEED)
    if kind in ("rsvd_full", "lanczos_full"):
        del A, b
        A = workloads.factor_rank_torch(65536, 16384, 2048, seed=SEED)

    def once():
        if kind == "lsr":
            return rmc.rmc_lsr_sketch(A, b, 1024, "countsketch", SEED)
        if kind == "lsr_precise":
            return rmc.rmc_lsr_precise(A, b, 1024, "countsketch", SEED, max_iters=4, tol=0.0)
        if kind == "rsvd":
            return rmc.rmc_rsvd(A, 100, 20, 1, SEED, prec=GAUSS_PREC)[1]
        if kind == "rsvd_full":
            return rmc.rmc_rsvd(A, 100, 20, int(os.environ.get("RMC_PROBE_Q", "0")), SEED, prec=GAUSS_PREC)[1]
        if kind == "lanczos_full":
            return rmc.rmc_block_lanczos(A, 100, 120, 2, SEED, prec=GAUSS_PREC)[1]
        prec = GAUSS_PREC if kind == "gaussian" else "fp32"
        return rmc.rmc_sketch(A, 1024, kind, SEED, prec=prec)

    for _ in range(2):
        once()
    rmc.rmc_sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(2):
        out = once()
    e1.record()
    rmc.rmc_sync()
    print(json.dumps({"probe": kind, "ms_per_call": e0.elapsed_time(e1) / 2, "checksum": float(out.double().sum())}))
    return 0


# Stop once a step changes z by at most this fraction of max|z| (the FP32 inputs make ~1e-13 the floor).
PRECISE_TOL = 1e-12


def precise_measure(torch, rmc, A, b, s=4096):
    """Machine-precision least squares (Algorithm 4.1) on the tall regression workload, every kind at s = 4096:
    call time, steps taken, and the residual + gradient pass over A as a roofline entry (algorithmic bytes
    per pass: A and b read once).  The error is the normal-equation residual ||A^T (b - A x)|| / (||A|| ||b||)
    evaluated in FP64 on the device, zero at the exact solution whatever the size."""
    m, n = A.shape
    pk = peaks()
    out = {"workload": "tall-lsr %dx%d, s=%d, tol %g, at most 60 steps" % (m, n, s, PRECISE_TOL), "calls": {}}
    A64 = A.double()
    b64 = b.double()
    anorm = float(torch.linalg.matrix_norm(A64, ord="fro"))
    bnorm = float(torch.linalg.vector_norm(b64))
    for kind in ("countsketch", "srht", "gaussian"):
        prec = GAUSS_PREC if kind == "gaussian" else "fp32"
        rmc.rmc_lsr_precise(A, b, s, kind, SEED, prec=prec, max_iters=60, tol=PRECISE_TOL)
        rmc.rmc_sync()
        rmc.rmc_profile_begin()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        x, it = rmc.rmc_lsr_precise(A, b, s, kind, SEED, prec=prec, max_iters=60, tol=PRECISE_TOL,
                                    want_iters=True)
        e1.record()
        rmc.rmc_sync()
        npass, pass_ms = rmc.rmc_profile_read(rmc.K_LSR_PASS)
        rmc.rmc_profile_end()
        steps = int(it.item())
        # launches after convergence return at once, so the pass time is spread over the steps that ran
        per_pass_bytes = 4.0 * (m * n + m)
        g = A64.T @ (b64 - A64 @ x)
        out["calls"][kind] = {
            "ms": e0.elapsed_time(e1), "steps": steps, "pass_launches": npass, "pass_ms_total": pass_ms,
            "pass_ms_per_step": pass_ms / max(1, steps),
            "pass_gbs": per_pass_bytes * steps / (pass_ms / 1e3) / 1e9 if steps else None,
            "pass_frac_hbm_of_measured": (per_pass_bytes * steps / (pass_ms / 1e3) / 1e9 / pk["hbm_gbs"]
                                          if steps else None),
            "normal_eq_residual": float(torch.linalg.vector_norm(g)) / (anorm * bnorm)}
    del A64, b64
    torch.cuda.empty_cache()
    return out


def lanczos_measure(torch, rmc, A, k=100, s=120, q=2):
    """Block Lanczos (Algorithm 5.1) on the large randomized-SVD workload: block size s, q blocks (2q passes)."""
    m, n = A.shape
    out = {"workload": "block lanczos %dx%d k=%d s=%d q=%d" % (m, n, k, s, q), "calls": {}}
    for prec in ("tf32", "fp32"):
        rmc.rmc_block_lanczos(A, k, s, q, SEED, prec=prec)
        rmc.rmc_sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        _, sigma, _ = rmc.rmc_block_lanczos(A, k, s, q, SEED, prec=prec)
        e1.record()
        rmc.rmc_sync()
        ms = e0.elapsed_time(e1)
        out["calls"][prec] = {"ms": ms, "passes": 2 * q, "hbm_gbs": 2 * q * 4.0 * m * n / ms / 1e6,
                              "sigma1": float(sigma[0]), "sigma100": float(sigma[-1])}
    return out


def gaussian_forms_measure(torch, rmc, A, b):
    """Whole SRHT and count-sketch calls on [A, b] (device time of every kernel of the call, algorithmic bytes
    against the HBM peak), then the Gaussian sketch of [A, b] in each operand precision (FP32 CUDA cores;
    TF32 and BF16 tensor cores) at s = 1024 and 4096: device time per call (three calls, CUDA events), TFLOP/s of
    the product 2 m (n + 1) s, and the relative Frobenius difference from the FP32 form's sketch (the FP32 form
    is pinned to the oracle at 1e-5 by the tests; TF32 and BF16 differ from it by their operand rounding)."""
    m, n = A.shape
    # [A, b] with a 16-byte row pitch, as the tensor-core and TMA paths need (a 257-float pitch would send every
    # form to the CUDA-core fallback)
    ld = (n + 1 + 3) // 4 * 4
    Abp = torch.empty(m, ld, device=A.device, dtype=A.dtype)
    Abp[:, :n] = A
    Abp[:, n] = b
    Ab = Abp[:, :n + 1]
    pk = peaks()
    out = {"workload": "tall-lsr %dx%d + b, Gaussian sketch of [A, b]" % (m, n), "calls": {}}
    # whole calls of the HBM-bound kinds (every kernel of the call, e.g. both SRHT stages), one call at a time
    for kind in ("srht", "countsketch"):
        for s in (1024, 4096):
            rmc.rmc_sketch(Ab, s, kind, SEED)
            rmc.rmc_sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(3):
                rmc.rmc_sketch(Ab, s, kind, SEED)
            e1.record()
            rmc.rmc_sync()
            ms = e0.elapsed_time(e1) / 3
            gbs = call_bytes(m, n, s) / ms / 1e6
            out["calls"]["%s_call_s%d" % (kind, s)] = {"ms": ms, "gbs": gbs, "frac_hbm": gbs / pk["hbm_gbs"]}
    for s in (1024, 4096):
        # the drawing bound: the same normals with no product (one CTA of 16 drawing warps per SM)
        rmc.rmc_gaussian_draw_floor(m, s, SEED)
        rmc.rmc_sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            rmc.rmc_gaussian_draw_floor(m, s, SEED)
        e1.record()
        rmc.rmc_sync()
        floor_ms = e0.elapsed_time(e1) / 3
        out["calls"]["draw_floor_s%d" % s] = {"ms": floor_ms, "normals_per_s": m * s / floor_ms * 1e3}
        ref = None
        for prec in ("fp32", "tf32", "bf16"):
            C = rmc.rmc_sketch(Ab, s, "gaussian", SEED, prec=prec)
            rmc.rmc_sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(3):
                C = rmc.rmc_sketch(Ab, s, "gaussian", SEED, prec=prec)
            e1.record()
            rmc.rmc_sync()
            ms = e0.elapsed_time(e1) / 3
            tflops = 2.0 * m * (n + 1) * s / ms / 1e9
            rec = {"ms": ms, "tflops": tflops}
            if prec == "fp32":
                ref = C.double()
                rec["frac_fp32_alu_peak"] = tflops / (152 * 128 * 2 * pk["sm_max_mhz"] * 1e6 / 1e12)
            else:
                ratio = 1.1 / 2.25 if prec == "tf32" else 1.0
                rec["frac_tensor_peak"] = tflops / (pk["bf16_tflops"] * ratio)
                rec["relfro_vs_fp32"] = float(torch.linalg.matrix_norm(C.double() - ref) /
                                              torch.linalg.matrix_norm(ref))
                rec["draw_floor_over_ms"] = floor_ms / ms   # 1.0: the sketch costs no more than drawing its normals
            out["calls"]["%s_s%d" % (prec, s)] = rec
    del Ab, Abp
    torch.cuda.empty_cache()
    return out


def rsvd_measure(torch, rmc):
    """The large randomized-SVD workload (A = G1 diag(1/i) G2^T, 65,536 x 16,384, rank 2048; k = 100, p = 20)
    at q = 0, 1, 2 in FP32, 3xTF32, TF32 and BF16 operands: device time per call and useful TFLOP/s of the
    products with A (2q + 2 passes of 2 m n l flops)."""
    import workloads
    m, n, k, p = 65536, 16384, 100, 20
    A = workloads.factor_rank_torch(m, n, 2048, seed=SEED)
    out = {"workload": "rsvd 65536x16384 rank-2048 sigma_i=1/i, k=100 p=20", "calls": {}}
    ref = {}
    for prec in ["fp32", "tf32x3", "tf32", "bf16"]:
        for q in [0, 1, 2]:
            rmc.rmc_rsvd(A, k, p, q, SEED, prec=prec)
            rmc.rmc_sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 1 if prec == "fp32" else 3
            e0.record()
            for _ in range(reps):
                _, sigma, _ = rmc.rmc_rsvd(A, k, p, q, SEED, prec=prec)
            e1.record()
            rmc.rmc_sync()
            ms = e0.elapsed_time(e1) / reps
            flops = (2 * q + 2) * 2.0 * m * n * (k + p)
            out["calls"]["%s_q%d" % (prec, q)] = {"ms": ms, "product_tflops": flops / ms / 1e9,
                                                  "hbm_gbs": (2 * q + 2) * 4.0 * m * n / ms / 1e6,
                                                  "frac_hbm_of_measured": (2 * q + 2) * 4.0 * m * n / ms / 1e6
                                                  / peaks()["hbm_gbs"],
                                                  "sigma1": float(sigma[0]), "sigma100": float(sigma[-1])}
            if prec == "fp32":
                ref[q] = sigma.double()
            else:
                # largest relative difference of the k singular values from the FP32-product form's
                out["calls"]["%s_q%d" % (prec, q)]["sigma_maxrel_vs_fp32"] = float(
                    ((sigma.double() - ref[q]).abs() / ref[q]).max())
    out["block_lanczos"] = lanczos_measure(torch, rmc, A)
    del A
    torch.cuda.empty_cache()
    return out


def matmul_peaks(torch):
    """Context figures: cuBLAS GEMM rates through torch.matmul (best of 5, CUDA events) in FP64, FP32 (no TF32),
    TF32 and BF16.  Library GEMMs, not part of the path; they show what each precision costs on this GPU."""
    out = {}
    for name, dtype, tf32, size in [("dgemm", torch.float64, False, 4096), ("sgemm", torch.float32, False, 8192),
                                    ("tf32_gemm", torch.float32, True, 8192), ("bf16_gemm", torch.bfloat16, False, 8192)]:
        prev = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = tf32
        try:
            a = torch.randn(size, size, device="cuda", dtype=torch.float32).to(dtype)
            b = torch.randn(size, size, device="cuda", dtype=torch.float32).to(dtype)
            torch.matmul(a, b)
            best = None
            for _ in range(5):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b)
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                best = ms if best is None else min(best, ms)
            out[name] = {"n": size, "ms": best, "tflops": 2.0 * size ** 3 / best / 1e9}
        finally:
            torch.backends.cuda.matmul.allow_tf32 = prev
        del a, b
    print(json.dumps({"probe": "peaks", "matmul": out}))
    return 0


def batch_measure(torch, rmc, count=4096, m_range=(512, 32768), reps=3):
    """The batched workload: ``count`` uneven problems (half rsvd k=16 p=8 q=1, half count-sketch least squares
    with s = 4n; m log-uniform on m_range, n uniform on [16, 256]) in one rmc_batch_run call.  Algorithmic
    bytes: the passes over A (2q + 2 for rsvd, one over [A, b] for least squares)."""
    import workloads
    specs = workloads.batch_specs(count=count, seed=SEED, m_range=m_range)
    reqs, keep, nbytes = [], [], 0
    for sp in specs:
        A, b = workloads.batch_problem_torch(sp)
        if sp["kind"] == "rsvd":
            r, o = rmc.rsvd_request(A, sp["k"], sp["p"], sp["q"], sp["seed"])
            nbytes += (2 + 2 * sp["q"]) * sp["m"] * sp["n"] * 4
        else:
            r, o = rmc.lsr_request(A, b, sp["s"], sp["seed"])
            nbytes += sp["m"] * (sp["n"] + 1) * 4
        reqs.append(r)
        keep.append((A, b, o))
    torch.cuda.synchronize()
    rmc.rmc_batch_run(reqs)
    rmc.rmc_sync()
    # the default schedule, then the autotuned one (tuned on this workload's own problems)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        rmc.rmc_batch_run(reqs)
    e1.record()
    rmc.rmc_sync()
    ms_default = e0.elapsed_time(e1) / reps
    default_tiles = rmc.rmc_batch_get_tiles()
    tiles = rmc.rmc_batch_autotune(reqs, reps=2)
    launches0 = rmc.rmc_launch_counter()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        rmc.rmc_batch_run(reqs)
    e1.record()
    rmc.rmc_sync()
    ms = e0.elapsed_time(e1) / reps
    launches = (rmc.rmc_launch_counter() - launches0) / reps
    rmc.rmc_profile_begin()
    rmc.rmc_batch_run(reqs)
    rmc.rmc_sync()
    _, kms = rmc.rmc_profile_read(rmc.K_BATCH)
    rmc.rmc_profile_end()
    hbm = peaks()["hbm_gbs"]
    out = {"workload": "%d problems: rsvd k=16 p=8 q=1 / countsketch lsr s=4n, m log-uniform %s, n U[16,256]"
                       % (count, list(m_range)),
           "ms": ms, "kernel_ms": kms, "problems_per_s": count / ms * 1e3, "bytes": nbytes,
           "gbs": nbytes / ms / 1e6, "kernel_gbs": nbytes / kms / 1e6, "frac_hbm_of_measured": nbytes / kms / 1e6 / hbm,
           "launches_per_call": launches, "ms_default_schedule": ms_default, "tile_table": tiles}
    rmc.rmc_batch_set_tiles(default_tiles)
    del keep
    torch.cuda.empty_cache()
    return out


def serve_measure(torch, rmc, rates=(100, 1000, 2500, 5000), window_s=2.0, pool=48, budget=64 << 30, nstreams=8,
                  max_outstanding=4096):
    """The served stream: Poisson arrivals at each rate for window_s seconds over a pool of resident problems
    (m log-uniform [1e3, 2e5], n log-uniform [32, 1024]; 60% count-sketch least squares with s = 4n, 40%
    randomized k-SVD with k in {8, 32, 64}, p = 8, q = 1), admitted under a 64 GB budget on nstreams streams.  The
    stream is replayed in real time, once with FP32 products and once with 3xTF32 products for the k-SVDs (the
    same 1e-4 singular-value tolerance against the oracle: equal stated error).  Reports completed requests/s
    and p50/p99 latency (submit to completion).  Load shedding: an arrival that finds max_outstanding requests
    queued or in flight is rejected and counted (their outputs hold device memory, so an overloaded stream would
    otherwise grow without bound).  Resident runs ("_resident"): every least-squares request on a problem shares
    that problem's sketch (seed = pool index) and brings one of four right-hand sides of the problem; the server
    keeps S^T A and its factor resident, so only the first request per problem sketches A."""
    import time
    import workloads
    ms_, ns_ = workloads.serve_pool(pool, seed=SEED)
    g = torch.Generator(device="cuda")
    g.manual_seed(SEED)
    mats = []
    for m, n in zip(ms_, ns_):
        A = torch.randn(m, n, generator=g, device="cuda", dtype=torch.float32)
        b = torch.randn(m, generator=g, device="cuda", dtype=torch.float32)
        mats.append((A, b))
    torch.cuda.synchronize()
    out = {"workload": "poisson stream, pool of %d resident problems m~logU[1e3,2e5] n~logU[32,1024]; 60%% lsr "
                       "(countsketch s=4n) / 40%% rsvd (k in {8,32,64}, p=8, q=1); budget 64 GB, %d streams"
                       % (pool, nstreams), "window_s": window_s, "runs": {}}
    # the resident variant: one sketch per problem (seed = pool index) and a fresh right-hand side per least-squares
    # request from a bank of four per problem; the server keeps S^T A and its factor resident (16 GB cap)
    rhs_bank = [[torch.randn(A.shape[0], generator=g, device="cuda", dtype=torch.float32) for _ in range(4)]
                for A, _ in mats]
    variants = [(prec, False, rate) for prec in ("fp32", "tf32x3") for rate in rates]
    variants += [(prec, True, rate) for prec in ("fp32", "tf32x3") for rate in rates if rate >= 2500]
    for prec, resident, rate in variants:
        arr = workloads.serve_arrivals(rate, window_s, pool, seed=SEED + rate)
        srv = rmc.Server(budget, nstreams=nstreams, max_batch=256)
        if resident:
            srv.resident(16 << 30)
        live, lat = {}, []
        rejected, failed, spec_of = 0, [], {}
        i, t0 = 0, time.perf_counter()
        while True:
            now = time.perf_counter() - t0
            while i < len(arr) and arr[i]["t"] <= now:
                a = arr[i]
                if len(live) >= max_outstanding:
                    rejected += 1
                    i += 1
                    continue
                A, b = mats[a["pool"]]
                n = A.shape[1]
                if a["kind"] == "lsr":
                    if resident:
                        b = rhs_bank[a["pool"]][a["seed"] % 4]
                    seed = a["pool"] if resident else a["seed"]
                    r, o = rmc.lsr_request(A, b, a["s_factor"] * n, seed)
                    tk = srv.submit(r, sketch="countsketch", prec="fp32")
                    spec_of[tk] = ("lsr", int(A.shape[0]), int(n), a["s_factor"] * n, a["seed"], a["pool"])
                else:
                    k = max(1, min(a["k"], n - a["p"]))
                    r, o = rmc.rsvd_request(A, k, a["p"], a["q"], a["seed"])
                    tk = srv.submit(r, prec=prec)
                    spec_of[tk] = ("rsvd", int(A.shape[0]), int(n), k, a["p"], a["q"], a["seed"], a["pool"])
                live[tk] = o
                i += 1
            srv.progress()
            for tk, st, l in srv.poll():
                if st != rmc.RMC_OK:
                    failed.append((st,) + spec_of[tk])
                else:
                    lat.append(l)
                del live[tk]
                del spec_of[tk]
            if i == len(arr) and not live:
                break
        t_end = time.perf_counter() - t0
        srv.close()
        lat_ms = np.sort(np.array(lat)) * 1e3
        out["runs"]["%s%s_rate%d" % (prec, "_resident" if resident else "", rate)] = {
            "offered_per_s": len(arr) / window_s, "completed": len(lat), "rejected": rejected,
            "failed": len(failed), "failed_first": failed[:8],
            "completed_per_s": len(lat) / t_end,
            "p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99)),
            "mean_ms": float(lat_ms.mean()), "drain_s": t_end}
    del mats, rhs_bank
    torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--probe", choices=["countsketch", "srht", "gaussian", "lsr", "lsr_precise", "rsvd", "rsvd_full", "lanczos_full",
                                        "batch", "peaks"], default=None,
                    help="run one small case of one kernel family (for profiler captures) and exit")
    ap.add_argument("--no-rsvd", action="store_true", help="skip the large randomized-SVD measurement")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-problems measurement")
    ap.add_argument("--no-serve", action="store_true", help="skip the served-stream measurement")
    ap.add_argument("--serve-only", action="store_true",
                    help="run only the served-stream measurement (with --serve-window / --serve-rates) and exit")
    ap.add_argument("--serve-window", type=float, default=2.0, help="seconds of Poisson arrivals per rate")
    ap.add_argument("--serve-rates", type=str, default="100,1000,2500,5000", help="offered rates, requests/s")
    ap.add_argument("--serve-streams", type=int, default=8, help="streams of the request server")
    args = ap.parse_args()
    if args.probe:
        return run_probe(args.probe)
    if args.serve_only:
        import torch
        import paper_1505_07570_gb300 as rmc
        rates = tuple(int(r) for r in args.serve_rates.split(","))
        print(json.dumps({"serve": serve_measure(torch, rmc, rates=rates, window_s=args.serve_window,
                                                 nstreams=args.serve_streams)}))
        return 0
    world, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    return run_ours(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
