"""Host-side sharding of the batched workload across ranks (no GPU): a disjoint,
balanced cover of the trains, identical on every rank, checked with two gloo ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2602_20226_gb300 import inputs
from paper_2602_20226_gb300.shard import gather_counts, lpt_partition, nominal_work


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
