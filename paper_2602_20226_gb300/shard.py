"""Split the data-parallel workloads across ranks (one GPU per rank).

The batched apply + round has no exchange step: every train is rounded on its own, so
the ranks only need a disjoint cover of the trains with balanced work.  `lpt_partition`
assigns trains largest-first to the least-loaded rank (the longest-processing-time rule)
by nominal rounding work, identically on every rank (a deterministic function of the
shapes); `gather_counts` collects the per-rank statistics once at the end.

Fitting a train to sample points shards the samples instead: each rank evaluates the train
and the adjoint of the evaluation on its own contiguous block of samples
(`sample_block`), and the one exchange of the step is the sum of the core gradients over
the ranks (`allreduce_core_grads`, a single all-reduce of the flattened cores; about 1.3 MB
in FP32 for a 40-site rank-64 train).
"""
from __future__ import annotations


def nominal_work(L: int, r: int, a: int, d: int = 2) -> float:
    """Nominal rounding work of one train of the uneven batch: its bonds have rank ~ a r,
    each costing ~ (a r)^3 (QR + SVD + GEMMs), times the L - 1 bonds."""
    n = float(a * r)
    return (L - 1) * n * n * n * d


def lpt_partition(shapes: list[tuple[int, int, int]], world: int) -> list[list[int]]:
    """Indices of the trains of each rank: largest nominal work first, each to the rank with
    the least work so far (ties to the lower rank).  Every train goes to exactly one rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(shapes)), key=lambda i: (-nominal_work(*shapes[i]), i))
    load = [0.0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        k = min(range(world), key=lambda j: (load[j], j))
        parts[k].append(i)
        load[k] += nominal_work(*shapes[i])
    return [sorted(p) for p in parts]


def gather_counts(values: list[float]):
    """All-gather of a few per-rank numbers (torch.distributed must be initialised)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor(values, dtype=torch.float64)
    if dist.get_backend() == "nccl":
        t = t.cuda()
    out = [torch.zeros_like(t) for _ in range(dist.get_world_size())]
    dist.all_gather(out, t)
    return [o.cpu().tolist() for o in out]


def sample_block(n: int, world: int, rank: int) -> tuple[int, int]:
    """[lo, hi) of this rank's samples: contiguous blocks whose sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world")
    q, r = divmod(int(n), world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def allreduce_core_grads(grads, group=None) -> None:
    """Sum the per-rank core gradients in place over all ranks (torch.distributed must be
    initialised): the cores are flattened into one buffer so the step costs one all-reduce."""
    import torch
    import torch.distributed as dist

    if not grads:
        return
    flat = torch.cat([g.reshape(-1) for g in grads])
    dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
    off = 0
    for g in grads:
        n = g.numel()
        g.copy_(flat[off:off + n].view_as(g))
        off += n


def aggregate_throughput(units: float, seconds: float, device=None, group=None) -> tuple[float, float]:
    """Whole-job throughput of a weakly scaled run: the units all ranks processed and the
    slowest rank's time (torch.distributed must be initialised).  Returns (total units,
    max seconds); the job's rate is their quotient."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(units), float(seconds)], dtype=torch.float64, device=device)
    tot = t.clone()
    dist.all_reduce(tot, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(tot[0].item()), float(t[1].item())
