"""Run one workload of the library from the command line (timing, ranks, profiling).

    python -m paper_2602_20226_gb300.cli --form fp64  --n-dims 2 --bits 20 --rank 64 --eps 1e-8
    python -m paper_2602_20226_gb300.cli --form mixed --n-dims 2 --bits 20 --rank 64 --eps 1e-6

Builds the seeded quantics TT (n_dims x bits sites, interleaved, d = 2, cores N(0, 1)
scaled by 1/sqrt(d r)), applies the Dirichlet Laplacian MPO of that grid (rank 3 in 1D,
5 in 2D, 7 in 3D) and rounds the result, `--repeat` times, printing the wall time of
each repetition and the output ranks.  `--op hadamard` rounds x (.) x instead.

    python -m paper_2602_20226_gb300.cli --batch 512 --form mixed --eps 1e-6

runs tt_apply_round_batched on the uneven batch instead: trains with L ~ U[20, 60],
ranks ~ U[8, 128], each with its own random MPO of rank 3..5 (seed 4).

    python -m paper_2602_20226_gb300.cli --eval 65536 --n-dims 2 --bits 20 --rank 64

times tt_eval and tt_eval_backward of the FP32 train (seed 230) at that many uniform index
tuples (seed 231), with CUDA events.

    python -m paper_2602_20226_gb300.cli --gemm 4096 --gemm-form sliced --repeat 10

times one FP32 tensor-core GEMM (N x N x N, N(0, 1) operands, seed 1) with CUDA events
and prints its TFLOP/s and its largest error against an FP64 product.
"""
from __future__ import annotations

import argparse
import time

import torch

from . import _abi, api, inputs, qtt


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(prog="python -m paper_2602_20226_gb300.cli")
    ap.add_argument("--form", choices=["fp64", "mixed"], default="fp64")
    ap.add_argument("--op", choices=["laplacian", "hadamard"], default="laplacian")
    ap.add_argument("--n-dims", type=int, default=2)
    ap.add_argument("--bits", type=int, default=20)
    ap.add_argument("--rank", type=int, default=64)
    ap.add_argument("--eps", type=float, default=1e-8)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--batch", type=int, default=0, help="trains of the uneven batch (0: one train)")
    ap.add_argument("--gemm", type=int, default=0, help="size N of one N x N x N FP32 GEMM to time (0: none)")
    ap.add_argument("--gemm-form", choices=["sliced", "tf32x3"], default="sliced")
    ap.add_argument("--eval", type=int, default=0, help="samples of tt_eval / tt_eval_backward to time (0: none)")
    a = ap.parse_args(argv)
    if a.batch > 0:
        return _batch(a)
    if a.gemm > 0:
        return _gemm(a)
    if a.eval > 0:
        return _eval(a)

    dtype = torch.float64 if a.form == "fp64" else torch.float32
    prec = _abi.TT_PREC_FP64 if a.form == "fp64" else _abi.TT_PREC_MIXED
    L = a.n_dims * a.bits
    X = api.TT.from_numpy(inputs.random_tt(a.seed, L, 2, a.rank), dtype=dtype)
    if a.op == "laplacian":
        W = api.MPO.from_numpy(qtt.laplacian_mpo(a.n_dims, a.bits), dtype=dtype)
        Y = api.tt_apply_mpo(W, X)
    else:
        Y = api.tt_hadamard(X, X)
    ws = torch.empty(api.tt_round_workspace_size(Y, prec), dtype=torch.uint8, device=X.device)
    for i in range(a.repeat):
        torch.cuda.synchronize()
        t = time.perf_counter()
        Z, nrm = api.tt_round(Y, a.eps, prec=prec, workspace=ws)
        torch.cuda.synchronize()
        print(f"[{i}] {a.form} {a.op} round: {(time.perf_counter() - t) * 1e3:.2f} ms, "
              f"max rank {max(Y.ranks)} -> {max(Z.ranks)}, norm {nrm:.12e}", flush=True)



def _batch(a) -> None:
    import numpy as np

    dtype = torch.float64 if a.form == "fp64" else torch.float32
    shapes = inputs.batch_shapes(4, a.batch)
    X = [api.TT.from_numpy([c.astype(np.float32) for c in inputs.random_tt(4000 + i, L, 2, r)], dtype=dtype)
         for i, (L, r, _) in enumerate(shapes)]
    W = [api.MPO.from_numpy([c.astype(np.float32) for c in inputs.random_mpo(4500 + i, L, 2, m)], dtype=dtype)
         for i, (L, _, m) in enumerate(shapes)]
    for i in range(a.repeat):
        torch.cuda.synchronize()
        t = time.perf_counter()
        outs = api.tt_apply_round_batched(W, X, a.eps)
        torch.cuda.synchronize()
        print(f"[{i}] {a.form} batch of {a.batch}: {(time.perf_counter() - t) * 1e3:.1f} ms, "
              f"max rank {max(max(o.ranks) for o in outs)}", flush=True)


def _eval(a) -> None:
    import numpy as np

    L, n = a.n_dims * a.bits, a.eval
    X = api.TT.from_numpy([c.astype(np.float32) for c in inputs.random_tt(230, L, 2, a.rank)], dtype=torch.float32)
    dg = torch.as_tensor(inputs.random_digits(231, n, [2] * L), device="cuda")
    dv = torch.as_tensor(np.random.default_rng(232).standard_normal(n).astype(np.float32), device="cuda")
    for i in range(a.repeat):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record()
        api.tt_eval(X, dg)
        e[1].record()
        api.tt_eval_backward(X, dg, dv)
        e[2].record()
        e[2].synchronize()
        print(f"[{i}] eval of {n} samples, L={L}, rank {a.rank}: forward {e[0].elapsed_time(e[1]):.3f} ms, "
              f"backward {e[1].elapsed_time(e[2]):.3f} ms", flush=True)


def _gemm(a) -> None:
    n = a.gemm
    g = torch.Generator(device="cuda").manual_seed(1)
    A = torch.randn(n, n, device="cuda", generator=g)
    B = torch.randn(n, n, device="cuda", generator=g)
    C = torch.empty(n, n, device="cuda")
    api.gemm_f32(A, B, C, form=a.gemm_form)  # first launch: configuration, not timed
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(a.repeat):
        api.gemm_f32(A, B, C, form=a.gemm_form)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.repeat
    ref = A.double() @ B.double()
    err = ((C.double() - ref).abs().max() / ref.abs().max()).item()
    print(f"{a.gemm_form} gemm n={n}: {ms:.3f} ms, {2.0 * n ** 3 / ms / 1e9:.1f} TFLOP/s, "
          f"max |C - AB| / max |AB| = {err:.2e}", flush=True)


if __name__ == "__main__":
    main()
