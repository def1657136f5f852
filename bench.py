#!/usr/bin/env python
"""Benchmark of the quantics-TT apply + round hot path on GB300.

One step = y = W x (MPO apply) followed by y' = round(y, eps) on one TT, all through
the libtt C ABI.  Default workload: 2D quantics TT, 2 x 20 bits interleaved (L = 40),
d = 2, rank 64 (seeded Gaussian cores), the 2D Dirichlet Laplacian MPO (rank 5,
pre-round rank 320), eps = 1e-8, the plain FP64 form.  Alongside, the same step in the
mixed form (FP32 cores; FP32 GEMMs with better-than-FP32 sums: the sliced tensor-core
form or compensated SIMT; FP32 bond SVDs with FP64 singular values and truncation), its
speed-up over FP64 and its error against the FP64 oracle, and the batched apply + round
of the uneven 512-train batch in both forms.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs an independent replica (a single TT's sweeps are a
sequential chain: replicas only); the reported value is the sum over ranks of the
work done divided by the slowest rank's time.
"""
from __future__ import annotations

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

METRIC = "MPO·TT apply+round GFLOP/s & % tensor peak, mixed vs FP64 GPU, rel err ≤1e-6"
MIXED_EPS = 1e-6
WORKLOAD = {
    "workload": "2D quantics TT L=40 (2x20 bits interleaved), d=2, rank 64, 2D Dirichlet Laplacian "
                "MPO rank 5 (n=320), apply + tt_round eps=1e-8",
    "L": 40, "bits": 20, "n_dims": 2, "rank": 64, "mpo_rank": 5, "eps": 1e-8, "seed": 2,
}
L2_FLUSH_BYTES = 512 << 20


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# FP64 ALU peak of GB300, derived from its unit count and clock: 152 SMs x 2 DFMA per
# clock per SM x 2 flops x 2.07 GHz = 1.26 TFLOP/s (a DFMA-loop microbenchmark measured
# 1.19 TFLOP/s at 2070 MHz).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = [r.split(",") for r in self.out.strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i]
                          and "Not" not in r[5 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def build_inputs(dtype):
    from paper_2602_20226_gb300 import inputs, qtt

    w = WORKLOAD
    x = inputs.random_tt(w["seed"], w["L"], 2, w["rank"])
    W = qtt.laplacian_mpo(w["n_dims"], w["bits"])
    if dtype == "f32":
        x = [c.astype(np.float32) for c in x]
        W = [c.astype(np.float32) for c in W]
    return x, W


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2602_20226_gb300 as tt
    from paper_2602_20226_gb300 import _abi
    from paper_2602_20226_gb300.flops import apply_flops, round_flops

    rank, world, local = _dist()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    lib = tt.load()
    eps = WORKLOAD["eps"]
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def make(dtype):
        x_np, W_np = build_inputs(dtype)
        tdt = torch.float64 if dtype == "f64" else torch.float32
        X = tt.TT.from_numpy(x_np, device=dev, dtype=tdt)
        W = tt.MPO.from_numpy(W_np, device=dev, dtype=tdt)
        Y0 = tt.tt_apply_mpo(W, X)
        ws = torch.empty(tt.tt_round_workspace_size(Y0, tt.TT_PREC_FP64 if dtype == "f64" else tt.TT_PREC_MIXED),
                         dtype=torch.uint8, device=dev)
        bufs = [torch.empty(c.numel(), dtype=tdt, device=dev) for c in Y0.cores]
        return x_np, W_np, X, W, ws, bufs

    def step(X, W, ws, bufs, prec, e=None):
        Y = tt.tt_apply_mpo(W, X)
        Z, _ = tt.tt_round(Y, eps if e is None else e, 0, prec, workspace=ws, out_buffers=bufs)
        return Y, Z

    def timed(X, W, ws, bufs, prec, K, Wm, e=None):
        for _ in range(Wm):
            step(X, W, ws, bufs, prec, e)
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        l0 = lib.tt_launch_count()
        ms_steps = []
        t0 = time.perf_counter()
        for _ in range(K):
            flush.zero_()  # L2 flush, outside the event-timed region
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            Y, Z = step(X, W, ws, bufs, prec, e)
            e1.record(stream)
            e1.synchronize()
            ms_steps.append(e0.elapsed_time(e1))
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - t0
        launches = int(lib.tt_launch_count() - l0)
        return Y, Z, ms_steps, wall, launches

    K, Wm = args.steps, args.warmup
    # ---- FP64 form (the reported value)
    x_np, W_np, X, W, ws, bufs = make("f64")
    with ClockSampler(dev.index or 0) as clk:
        Y, Z, ms64, wall64, launches = timed(X, W, ws, bufs, tt.TT_PREC_FP64, K, Wm)
    clocks = clk.summary()
    ms_step = float(np.mean(ms64))
    fl_apply = apply_flops([int(v) for v in W.ranks], X.ranks, X.dims)
    fl_round = round_flops(Y.ranks, Z.ranks, X.dims)
    flops_step = fl_apply + fl_round["total"]

    # ---- dominant kernel and its live event timing (one profiled step, same stream)
    lib.tt_profile_enable(1)
    step(X, W, ws, bufs, tt.TT_PREC_FP64)
    torch.cuda.synchronize(dev)
    prof = {}
    import ctypes
    for cls, name in [(0, "jacobi_svd"), (1, "householder_qr"), (2, "core_gemm"), (3, "certificate")]:
        ms_c, fl_c, n_c, ex_c = ctypes.c_double(), ctypes.c_double(), ctypes.c_uint64(), ctypes.c_double()
        lib.tt_profile_read(cls, ctypes.byref(ms_c), ctypes.byref(fl_c), ctypes.byref(n_c))
        lib.tt_profile_read_executed(cls, ctypes.byref(ex_c))
        prof[name] = {"ms": ms_c.value, "nominal_flops": fl_c.value, "executed_flops": ex_c.value,
                      "launches": int(n_c.value)}
    lib.tt_profile_enable(0)
    dom = max(prof, key=lambda k: prof[k]["ms"])
    d = prof[dom]
    # the roofline is taken on the executed work (the nominal SVD count charges 12 p^3 to
    # every bond, including those whose SVD the full-rank certificate skips)
    achieved_tflops = d["executed_flops"] / (d["ms"] * 1e-3) / 1e12 if d["ms"] > 0 else 0.0
    roofline = {
        "kernel": dom,
        "bound": "alu",
        "achieved": round(achieved_tflops, 6),
        "peak": round(FP64_PEAK_TFLOPS, 4),
        "unit": "TFLOP/s",
        "frac": round(achieved_tflops / FP64_PEAK_TFLOPS, 6),
        "traffic": None,
        "work": "executed flops (Jacobi: 6 p^3 per sweep that ran; QR: 4 m n^2 - 4 n^3 / 3; GEMM: 2 m n k)",
        "peak_source": "derived FP64 ALU peak (152 SMs x 2 DFMA/clk x 2 x 2.07 GHz)",
        "share_of_step": round(d["ms"] / max(ms_step, 1e-9), 4),
        "launch_ms_avg": round(d["ms"] / max(d["launches"], 1), 4),
        "phases": {k: {"ms": round(v["ms"], 3), "launches": v["launches"],
                       "nominal_tflops": round(v["nominal_flops"] / max(v["ms"], 1e-9) / 1e9, 4),
                       "executed_tflops": round(v["executed_flops"] / max(v["ms"], 1e-9) / 1e9, 4),
                       "frac_of_fp64_peak": round(v["executed_flops"] / max(v["ms"], 1e-9) / 1e9
                                                  / FP64_PEAK_TFLOPS, 4)}
                   for k, v in prof.items()},
    }
    # executed work of the whole step: the nominal count with the SVD term replaced by the
    # sweeps that ran, plus the certificates
    executed_step = flops_step - fl_round["svd"] + prof["jacobi_svd"]["executed_flops"] + \
        prof["certificate"]["executed_flops"]

    # ---- mixed form on the same TT shape (FP32 cores) against the FP64 form, both at
    # eps = 1e-6 (FP32 factors cannot resolve the 1e-8 of the main line)
    _, _, ms64m, _, _ = timed(X, W, ws, bufs, tt.TT_PREC_FP64, K, Wm, MIXED_EPS)
    ms_fp64_same_eps = float(np.mean(ms64m))
    x32, W32, X32, Wd32, ws32, bufs32 = make("f32")
    Y32, Z32, ms32, _, _ = timed(X32, Wd32, ws32, bufs32, tt.TT_PREC_MIXED, K, Wm, MIXED_EPS)
    ms_mixed = float(np.mean(ms32))

    # ---- secondary workloads (reported beside the main line)
    extra = {}
    if not args.no_extra:
        extra["batched"] = bench_batched(tt, dev, Wm, n_tt=args.batch_trains, rank=rank, world=world)
        extra["eval"] = bench_eval(tt, dev)
        extra["small_1d"] = bench_small(tt, dev)
        extra["grouped_2d"] = bench_grouped(tt, dev)
        extra["laplacian3d_rank256"] = bench_large(tt, dev, "laplacian3d")
        if args.large:
            extra["hadamard_square_rank64"] = bench_large(tt, dev, "hadamard")

    # ---- end to end: pinned host cores in, rounded cores out, through the public API
    xh = [torch.as_tensor(c).pin_memory() for c in x_np]
    wh = [torch.as_tensor(c).pin_memory() for c in W_np]
    h2d = sum(t.numel() * t.element_size() for t in xh + wh)
    e2e_ms, d2h = [], 0
    for it in range(Wm + K):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        Xd = tt.TT([t.to(dev, non_blocking=True) for t in xh])
        Wdd = tt.MPO([t.to(dev, non_blocking=True) for t in wh])
        Yd = tt.tt_apply_mpo(Wdd, Xd)
        Zd, _ = tt.tt_round(Yd, eps, 0, tt.TT_PREC_FP64, workspace=ws, out_buffers=bufs)
        outs = [c.to("cpu") for c in Zd.cores]
        e1.record(stream)
        e1.synchronize()
        if it >= Wm:
            e2e_ms.append(e0.elapsed_time(e1))
            d2h = sum(o.numel() * o.element_size() for o in outs)

    # ---- aggregate over ranks (replicas)
    t_max = ms_step
    if world > 1:
        tt_ = torch.tensor([ms_step], device=dev)
        dist.all_reduce(tt_, op=dist.ReduceOp.MAX)
        t_max = float(tt_.item())
    value = world * flops_step / (t_max * 1e-3) / 1e9
    flops_mixed = fl_apply + round_flops(Y32.ranks, Z32.ranks, X.dims)["total"]
    value_mixed = flops_mixed / (ms_mixed * 1e-3) / 1e9
    e2e_val = world * flops_step / (float(np.mean(e2e_ms)) * 1e-3) / 1e9

    err_mixed = None
    cpu = None
    if rank == 0:
        from oracle import core as ocore

        # accuracy of the mixed form against the FP64 oracle on the same FP32 inputs
        y32 = [c.astype(np.float64) for c in Y32.numpy()]
        ref32 = ocore.round_tt(y32, MIXED_EPS)
        err_mixed = ocore.rel_err(Z32.numpy(), ref32)
        if world == 1 and not args.no_cpu_baseline:
            cpu = cpu_baseline(x_np, W_np, eps, flops_step)
    if world > 1:
        dist.barrier()
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 4), "unit": "GFLOP/s", "n_gpus": world,
            "steps": K, "warmup": Wm, "ms_per_step": round(t_max, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(WORKLOAD, form="fp64", l2="flushed between steps (512 MB write, untimed)",
                           parallelism=f"replicas x{world}"),
            "nominal_flops_per_step": flops_step,
            "executed_flops_per_step": executed_step,
            "value_executed": round(world * executed_step / (t_max * 1e-3) / 1e9, 4),
            "round_flops": fl_round, "apply_flops": fl_apply,
            "ranks_out_max": max(Z.ranks),
            "mixed": {"value": round(value_mixed, 4), "unit": "GFLOP/s", "ms_per_step": round(ms_mixed, 4),
                      "eps": MIXED_EPS, "fp64_ms_per_step_same_eps": round(ms_fp64_same_eps, 4),
                      "dtype": "f32 cores; FP32 GEMMs with better-than-FP32 sums (sliced tensor-core form where its tiles fill the GPU, Dot2 SIMT below); FP64 full-rank certificate, else FP32 Jacobi; FP64 sigma/truncation/norm",
                      "speedup_vs_fp64": round(ms_fp64_same_eps / ms_mixed, 3),
                      "rel_err_vs_fp64_oracle": err_mixed},
            "roofline": roofline,
            "e2e": {"value": round(e2e_val, 4), "unit": "GFLOP/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": round(float(np.mean(e2e_ms)), 4)},
            "secondary": extra,
            "gpu_launches": launches,
            "gpu_launches_per_step": launches // max(K, 1),
            "clocks": clocks,
            "cpu_baseline": cpu,
            "wall_s_timed_region": round(wall64, 3),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _e_from_inner(a, b):
    """e(a, b) = |a - b| / |b| from the oracle's FP64 inner products.  Cheaper than the
    block-sum QR of core.rel_err on bonds of 640; the cancellation limits it to ~2e-7."""
    from oracle import core as ocore

    aa, bb, ab = ocore.inner(a, a), ocore.inner(b, b), ocore.inner(a, b)
    return float(np.sqrt(max(aa + bb - 2.0 * ab, 0.0) / bb))


def bench_batched(tt, dev, warm, n_tt=512, nstreams=5, repeats=3, rank=0, world=1):
    """Uneven batch (L ~ U[20,60], rank ~ U[8,128], MPO rank ~ U{3,4,5}), eps = 1e-6, through
    tt_apply_round_batched (lock-step over the trains): the mixed form (FP32 cores) against
    the FP64 form on the same trains, `repeats` timed calls per form, and the mixed results'
    error against the oracle on a sample that spans the cost range (cheapest, quartiles and
    the two most expensive trains).  Under torchrun every rank rounds its share of the trains
    (longest-processing-time split, no exchange); the value is all ranks' nominal flops over
    the slowest rank's time."""
    import torch
    import torch.distributed as dist

    from oracle import core as ocore
    from paper_2602_20226_gb300 import inputs
    from paper_2602_20226_gb300.flops import apply_flops, round_flops
    from paper_2602_20226_gb300.shard import aggregate_throughput, lpt_partition

    all_shapes = inputs.batch_shapes(4, n_tt)
    mine = lpt_partition(all_shapes, world)[rank]
    xs = [inputs.random_tt(4000 + i, all_shapes[i][0], 2, all_shapes[i][1]) for i in mine]
    ws = [inputs.random_mpo(4500 + i, all_shapes[i][0], 2, all_shapes[i][2]) for i in mine]
    streams = [torch.cuda.Stream(device=dev) for _ in range(nstreams)]
    res = {}
    outs_by_form = {}
    for form, dt in (("fp64", torch.float64), ("mixed", torch.float32)):
        X = [tt.TT.from_numpy([c.astype(np.float32) for c in x], device=dev, dtype=dt) for x in xs]
        W = [tt.MPO.from_numpy([c.astype(np.float32) for c in w], device=dev, dtype=dt) for w in ws]
        tt.tt_apply_round_batched(W[:8], X[:8], 1e-6, nstreams=nstreams, streams=streams)  # warm-up
        torch.cuda.synchronize(dev)
        secs = []
        for _ in range(repeats):
            if world > 1:
                dist.barrier()
            t0 = time.perf_counter()
            outs = tt.tt_apply_round_batched(W, X, 1e-6, nstreams=nstreams, streams=streams)
            torch.cuda.synchronize(dev)
            secs.append(time.perf_counter() - t0)
        sec = float(np.median(secs))
        flops = 0.0
        for x, w, o in zip(X, W, outs):
            yr = [a * b for a, b in zip(w.ranks, x.ranks)]
            flops += apply_flops(w.ranks, x.ranks, x.dims) + round_flops(yr, o.ranks, x.dims)["total"]
        if world > 1:
            flops, sec = aggregate_throughput(flops, sec, device=dev)
        res[form] = {"value": round(flops / sec / 1e9, 3), "unit": "GFLOP/s", "seconds": round(sec, 3),
                     "seconds_each": [round(v, 3) for v in secs], "nominal_flops": flops}
        outs_by_form[form] = outs
    # error of the mixed results against the oracle (inputs are the FP32 values in FP64), on
    # trains across the cost range
    order = sorted(range(len(mine)),
                   key=lambda q: all_shapes[mine[q]][0] * (all_shapes[mine[q]][1] * all_shapes[mine[q]][2]) ** 3)
    nq = len(order)
    picks = sorted({order[0], order[nq // 4], order[nq // 2], order[(3 * nq) // 4], order[max(nq - 2, 0)],
                    order[nq - 1]})
    errs, shapes, ranks_eq = [], [], []
    for q in picks:
        x64 = [c.astype(np.float32).astype(np.float64) for c in xs[q]]
        w64 = [c.astype(np.float32).astype(np.float64) for c in ws[q]]
        ref = ocore.round_tt(ocore.apply_mpo(w64, x64), 1e-6)
        got = outs_by_form["mixed"][q].numpy()
        errs.append(_e_from_inner(got, ref))
        shapes.append(list(all_shapes[mine[q]]))
        ranks_eq.append(ocore.ranks(got) == ocore.ranks(ref))
    return {"workload": f"{n_tt} trains, L~U[20,60], rank~U[8,128], MPO rank~U{{3,4,5}}, eps=1e-6, "
                        f"lock-step batched driver (host-timed, median of {repeats} calls)",
            "mixed": res["mixed"], "fp64": res["fp64"],
            "speedup_mixed_vs_fp64": round(res["fp64"]["seconds"] / res["mixed"]["seconds"], 3),
            "mixed_rel_err_vs_oracle_max": max(errs) if errs else None,
            "mixed_rel_err_vs_oracle_median": float(np.median(errs)) if errs else None,
            "mixed_err_sample": {"trains_L_rank_mpo_rank": shapes, "e": errs, "ranks_equal": ranks_eq,
                                 "choice": "cheapest, quartiles and the two most expensive trains by L (r a)^3",
                                 "metric": "(|a|^2+|b|^2-2<a,b>)^(1/2)/|b|, FP64 oracle inner products "
                                           "(resolution ~2e-7), b = oracle apply+round at eps=1e-6"}}


def bench_eval(tt, dev, n=1 << 20, L=40, r=64):
    """Evaluation at 2^20 index tuples, L = 40, rank 64, FP32 (samples/s and GFLOP/s)."""
    import torch

    from paper_2602_20226_gb300 import inputs
    from paper_2602_20226_gb300.flops import eval_flops

    x = tt.TT.from_numpy([c.astype(np.float32) for c in inputs.random_tt(230, L, 2, r)], device=dev,
                         dtype=torch.float32)
    dg = torch.as_tensor(inputs.random_digits(231, n, [2] * L), device=dev)
    out = torch.empty(n, dtype=torch.float32, device=dev)
    for _ in range(3):
        tt.tt_eval(x, dg, out=out)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    reps = 5
    e0.record()
    for _ in range(reps):
        tt.tt_eval(x, dg, out=out)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / reps
    fl = eval_flops(x.ranks, n)
    # the adjoint of the evaluation (gradient w.r.t. the cores) on the same samples
    dv = torch.as_tensor(np.random.default_rng(232).standard_normal(n).astype(np.float32), device=dev)
    tt.tt_eval_backward(x, dg, dv)
    torch.cuda.synchronize(dev)
    b0 = torch.cuda.Event(enable_timing=True)
    b1 = torch.cuda.Event(enable_timing=True)
    b0.record()
    tt.tt_eval_backward(x, dg, dv)
    b1.record()
    b1.synchronize()
    ms_b = b0.elapsed_time(b1)
    return {"workload": f"tt_eval, {n} samples, L={L}, rank {r}, FP32", "ms": round(ms, 3),
            "samples_per_s": round(n / (ms * 1e-3), 1), "value": round(fl / (ms * 1e-3) / 1e9, 2),
            "unit": "GFLOP/s",
            "backward": {"ms": round(ms_b, 3), "samples_per_s": round(n / (ms_b * 1e-3), 1),
                         "value": round(3 * fl / (ms_b * 1e-3) / 1e9, 2), "unit": "GFLOP/s",
                         "flops": "3x the forward: prefix sweep, suffix sweep, per-site sums",
                         "what": "tt_eval_backward (gradient w.r.t. the cores): FP32 prefix/suffix states "
                                 "and per-site sums over 2048-sample slices, FP64 across slices"}}


def bench_grouped(tt, dev, reps=3):
    """The 2D workload in the grouped-digit layout: the digits (x_q, y_q) of each scale on one
    core of mode 4 (L = 20, rank 64, FP64), the grouped Laplacian MPO (rank 5), apply + round
    at 1e-8; median of three calls after one warm-up, host-timed with device syncs."""
    import torch

    from paper_2602_20226_gb300 import inputs, qtt
    from paper_2602_20226_gb300.flops import apply_flops, round_flops

    X = tt.TT.from_numpy(inputs.random_tt(2, 20, 4, 64), device=dev)
    W = tt.MPO.from_numpy(qtt.group_mpo_sites(qtt.laplacian_mpo(2, 20), 2), device=dev)
    ts = []
    for i in range(reps + 1):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        Y = tt.tt_apply_mpo(W, X)
        Z, _ = tt.tt_round(Y, 1e-8)
        torch.cuda.synchronize(dev)
        if i:
            ts.append(time.perf_counter() - t0)
    sec = float(np.median(ts))
    fl = apply_flops([int(v) for v in W.ranks], X.ranks, X.dims) + round_flops(Y.ranks, Z.ranks, X.dims)["total"]
    return {"workload": "2D quantics TT, grouped digits (x_q, y_q) per core: L=20, d=4, rank 64, FP64, "
                        "grouped Laplacian MPO rank 5, apply + tt_round eps=1e-8 (median of 3 host-timed calls)",
            "ms": round(sec * 1e3, 3), "value": round(fl / sec / 1e9, 2), "unit": "GFLOP/s",
            "ranks_in_max": max(Y.ranks), "ranks_out_max": max(Z.ranks)}


def bench_large(tt, dev, case):
    """One of the two large configurations, one call each (apply or Hadamard product, then
    tt_round), host-timed with a device synchronisation on both sides:
      laplacian3d: 3D quantics TT (3 x 16 bits interleaved, L = 48), rank 256, FP32 cores,
          3D Dirichlet Laplacian MPO (rank 7, bond ranks 1792), mixed rounding at 1e-6;
      hadamard: 2D (2 x 20 bits, L = 40), rank 64, FP64, x (.) x (bond ranks 4096), FP64
          rounding at 1e-8.
    Checked on the GPU alone: the rounding bound ||z - y|| <= eps ||y|| from FP64 inner
    products (laplacian3d; at 1e-8 that difference is below the resolution of inner products)
    and the closed-form rank bound r (r + 1) / 2 of x (.) x.  The same workloads at L = 24 are
    checked against stored oracle values in the GPU tests."""
    import torch

    from paper_2602_20226_gb300 import inputs, qtt
    from paper_2602_20226_gb300.flops import apply_flops, hadamard_flops, round_flops

    if case == "laplacian3d":
        L, r, eps = 48, 256, 1e-6
        X = tt.TT.from_numpy([c.astype(np.float32) for c in inputs.random_tt(2, L, 2, r)], device=dev,
                             dtype=torch.float32)
        W = tt.MPO.from_numpy(qtt.laplacian_mpo(3, L // 3), device=dev, dtype=torch.float32)
    else:
        L, r, eps = 40, 64, 1e-8
        X = tt.TT.from_numpy(inputs.random_tt(2, L, 2, r), device=dev)
        W = None
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    Y = tt.tt_apply_mpo(W, X) if W is not None else tt.tt_hadamard(X, X)
    Z, _ = tt.tt_round(Y, eps)
    torch.cuda.synchronize(dev)
    sec = time.perf_counter() - t0
    fl = (apply_flops([int(v) for v in W.ranks], X.ranks, X.dims) if W is not None
          else hadamard_flops(X.ranks, X.ranks, X.dims)) + round_flops(Y.ranks, Z.ranks, X.dims)["total"]
    out = {"seconds": round(sec, 3), "value": round(fl / sec / 1e9, 2), "unit": "GFLOP/s",
           "ranks_in_max": max(Y.ranks), "ranks_out_max": max(Z.ranks), "eps": eps}
    if W is not None:
        out["workload"] = ("3D quantics TT L=48 (3x16 bits), rank 256, FP32 cores, 3D Dirichlet Laplacian MPO "
                           "rank 7, apply + tt_round mixed eps=1e-6 (one host-timed call)")
        zz, yy, zy = tt.tt_inner(Z, Z), tt.tt_inner(Y, Y), tt.tt_inner(Z, Y)
        out["rounding_rel_err"] = float(np.sqrt(max(zz + yy - 2.0 * zy, 0.0) / yy))
    else:
        out["workload"] = ("2D quantics TT L=40 (2x20 bits), rank 64, FP64, Hadamard square x*x (ranks 4096) "
                           "+ tt_round eps=1e-8 (one host-timed call)")
        out["closed_form_rank_bound"] = r * (r + 1) // 2
    return out


def bench_small(tt, dev, reps=50):
    """The small 1D workload: L = 10, rank 8, second-difference MPO (rank 3), eps = 1e-10,
    FP64 - latency of one apply + round (launch- and synchronisation-bound)."""
    import torch

    from paper_2602_20226_gb300 import inputs, qtt

    X = tt.TT.from_numpy(inputs.random_tt(1, 10, 2, 8), device=dev)
    W = tt.MPO.from_numpy(qtt.second_difference_mpo(10), device=dev)
    ws = torch.empty(1 << 20, dtype=torch.uint8, device=dev)
    ts = []
    lib = tt.load()
    n0 = lib.tt_launch_count()
    for i in range(reps + 5):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        Y = tt.tt_apply_mpo(W, X)
        Z, _ = tt.tt_round(Y, 1e-10, workspace=ws)
        torch.cuda.synchronize(dev)
        if i >= 5:
            ts.append((time.perf_counter() - t0) * 1e6)
    launches = (lib.tt_launch_count() - n0) / (reps + 5)
    return {"workload": "1D quantics TT L=10, rank 8, second-difference MPO rank 3, apply + tt_round "
                        "eps=1e-10, FP64 (host-timed, median of 50)",
            "us_per_step": round(float(np.median(ts)), 1), "us_min": round(float(np.min(ts)), 1),
            "launches_per_step": launches, "ranks_out": Z.ranks}


def cpu_baseline(x_np, W_np, eps, flops_step, repeats=2):
    """The FP64 oracle (numpy + LAPACK) on the host cores: full apply + round steps."""
    from oracle import core as ocore
    from oracle import structured

    W = structured.laplacian_mpo(WORKLOAD["n_dims"], WORKLOAD["bits"])
    times = []
    for _ in range(repeats):
        t0 = time.perf_counter()
        y = ocore.apply_mpo(W, [c.astype(np.float64) for c in x_np])
        ocore.round_tt(y, eps)
        times.append(time.perf_counter() - t0)
    s = float(np.mean(times))
    out = {"value": round(flops_step / s / 1e9, 4), "unit": "GFLOP/s", "cores": len(os.sched_getaffinity(0)),
           "kind": "oracle", "sample": f"{repeats} full steps (apply + round of the L=40 rank-64 TT), "
                                       f"{s:.2f} s each, numpy/LAPACK FP64"}
    s1 = _oracle_step_seconds_one_thread()
    if s1 is not None:
        out["one_thread"] = {"value": round(flops_step / s1 / 1e9, 4), "unit": "GFLOP/s", "cores": 1,
                             "sample": f"1 full step in a child process with one BLAS/OpenMP thread, {s1:.2f} s"}
    return out


def _oracle_step_seconds_one_thread():
    """One oracle step in a fresh child interpreter whose BLAS and OpenMP pools have one thread."""
    code = (
        "import time, sys\n"
        f"sys.path.insert(0, {ROOT!r})\n"
        "from oracle import core, structured\n"
        "from paper_2602_20226_gb300 import inputs\n"
        f"w = {dict(WORKLOAD)!r}\n"
        "x = inputs.random_tt(w['seed'], w['L'], 2, w['rank'])\n"
        "W = structured.laplacian_mpo(w['n_dims'], w['bits'])\n"
        "t0 = time.perf_counter()\n"
        "core.round_tt(core.apply_mpo(W, x), w['eps'])\n"
        "print(time.perf_counter() - t0)\n"
    )
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = "1"
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
        return float(r.stdout.strip().splitlines()[-1]) if r.returncode == 0 else None
    except (subprocess.TimeoutExpired, ValueError, IndexError):
        return None


def run_reference(args):
    """The oracle as the reference arm: timed on the host cores, same workload and metric."""
    rank, world, _ = _dist()
    if rank != 0:
        return
    from oracle import core as ocore
    from oracle import structured
    from paper_2602_20226_gb300.flops import apply_flops, round_flops

    x_np, _ = build_inputs("f64")
    W = structured.laplacian_mpo(WORKLOAD["n_dims"], WORKLOAD["bits"])
    eps = WORKLOAD["eps"]
    y = ocore.apply_mpo(W, x_np)
    z = ocore.round_tt(y, eps)
    flops = apply_flops(ocore.ranks(W), ocore.ranks(x_np), ocore.dims(x_np)) + \
        round_flops(ocore.ranks(y), ocore.ranks(z), ocore.dims(x_np))["total"]
    for _ in range(args.warmup):
        ocore.round_tt(ocore.apply_mpo(W, x_np), eps)
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        ocore.round_tt(ocore.apply_mpo(W, x_np), eps)
        ts.append(time.perf_counter() - t0)
    ms = float(np.mean(ts)) * 1e3
    val = flops / (ms * 1e-3) / 1e9
    cores = len(os.sched_getaffinity(0))
    line = {
        "impl": "reference", "metric": METRIC, "value": round(val, 4), "unit": "GFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(WORKLOAD, form="fp64 oracle (numpy/LAPACK, host cores)"),
        "cpu_baseline": {"value": round(val, 4), "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
                         "sample": "each step is one full apply + round of the workload"},
        "e2e": {"value": round(val, 4), "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the secondary workloads")
    ap.add_argument("--large", action="store_true",
                    help="also time x (.) x of the rank-64 2D train (bond ranks 4096; ~100 s)")
    ap.add_argument("--batch-trains", type=int, default=512,
                    help="trains in the secondary batched workload (default: the full batch of 512)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
