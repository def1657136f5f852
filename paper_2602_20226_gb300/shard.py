"""Split a batch of independent trains across ranks (one GPU per rank).

The batched apply + round has no exchange step: every train is rounded on its own, so
the ranks only need a disjoint cover of the trains with balanced work.  `lpt_partition`
assigns trains largest-first to the least-loaded rank (the longest-processing-time rule)
by nominal rounding work, identically on every rank (a deterministic function of the
shapes); `gather_counts` collects the per-rank statistics once at the end.
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
