"""Host-side sharding of the batched workload across ranks (no GPU): a disjoint,
balanced cover of the trains, identical on every rank, checked with two gloo ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2602_20226_gb300 import inputs
from paper_2602_20226_gb300.shard import (allreduce_core_grads, gather_counts, lpt_partition, nominal_work,
                                          sample_block)


def test_lpt_partition_cover_and_balance():
    shapes = inputs.batch_shapes(4, 64)
    for world in (1, 2, 3, 8):
        parts = lpt_partition(shapes, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(64))
        loads = [sum(nominal_work(*shapes[i]) for i in p) for p in parts]
        biggest = max(nominal_work(*s) for s in shapes)
        # LPT: the spread of the loads never exceeds the largest single job
        assert max(loads) - min(loads) <= biggest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    shapes = inputs.batch_shapes(4, 32)
    mine = lpt_partition(shapes, world)[rank]
    work = sum(nominal_work(*shapes[i]) for i in mine)
    got = gather_counts([float(len(mine)), work, float(sum(mine))])
    if rank == 0:
        q.put(got)
    dist.destroy_process_group()


def test_two_gloo_ranks_cover_the_batch():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    shapes = inputs.batch_shapes(4, 32)
    assert sum(g[0] for g in got) == 32
    assert sum(g[2] for g in got) == sum(range(32))  # disjoint cover (with the count above)
    total = sum(nominal_work(*s) for s in shapes)
    assert sum(g[1] for g in got) == pytest.approx(total)


def test_sample_blocks_cover():
    for n in (0, 1, 7, 1 << 20):
        for world in (1, 2, 3, 8):
            blocks = [sample_block(n, world, r) for r in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == n
            assert all(blocks[i][1] == blocks[i + 1][0] for i in range(world - 1))
            sizes = [b - a for a, b in blocks]
            assert max(sizes) - min(sizes) <= 1


def _fit_rank_main(rank, world, port, q):
    """Each rank: the fit-loss gradient on its block of samples (1/N of the global N), then
    the all-reduce; rank 0 reports the summed gradient."""
    import numpy as np
    import torch
    import torch.distributed as dist

    from oracle import grad

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    L, n = 12, 3000
    x = inputs.random_tt(71, L, 2, 5)
    dg = inputs.random_digits(72, n, [2] * L)
    f = inputs.fit_targets(dg, 6)
    lo, hi = sample_block(n, world, rank)
    v = __import__("oracle.core", fromlist=["evaluate"]).evaluate(x, dg[lo:hi])
    part = grad.evaluate_vjp(x, dg[lo:hi], (v - f[lo:hi]) / n)
    gt = [torch.from_numpy(np.ascontiguousarray(g)) for g in part]
    allreduce_core_grads(gt)
    if rank == 0:
        q.put([g.numpy() for g in gt])
    dist.destroy_process_group()


def test_two_gloo_ranks_sum_the_fit_gradient():
    """Sample-sharded fit gradient + one all-reduce == the gradient over all samples."""
    import numpy as np

    from oracle import grad

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_fit_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    L, n = 12, 3000
    x = inputs.random_tt(71, L, 2, 5)
    dg = inputs.random_digits(72, n, [2] * L)
    ref = grad.fit_loss_grad(x, dg, inputs.fit_targets(dg, 6))
    for a, b in zip(got, ref):
        assert np.abs(a - b).max() <= 1e-14 * max(1.0, np.abs(b).max())


def _agg_rank_main(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2602_20226_gb300.shard import aggregate_throughput

    # rank r processed 10 (r + 1) units in 2 + 3 r seconds
    got = aggregate_throughput(10.0 * (rank + 1), 2.0 + 3.0 * rank)
    q.put((rank, got))
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_throughput():
    """The bench's whole-job rate: units summed over the ranks, time of the slowest rank,
    the same on every rank."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_agg_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got[0] == got[1] == (30.0, 5.0)
