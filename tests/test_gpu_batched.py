"""Batched apply + round over trains of uneven length and rank (tt_apply_round_batched).

Every train of the batch is checked against the oracle's apply + round on the same
seeded inputs: FP64 form e <= 1e-12 with equal ranks; mixed form (FP32 cores) at the
error stated for that form (<= 4e-6 at eps = 1e-6 on 20..60-site trains; <= 2e-6 on the
short ragged batch).  The batched mixed form factors its Householder panels in FP64, which
brought the sampled trains of the 512-train batch from 1.4..1.9e-6 to 5.8e-7..9.7e-7 of
the unrounded trains; the bounds here date from the FP32 panels.
"""
import numpy as np
import pytest
import torch

from oracle import core
from paper_2602_20226_gb300 import inputs

pytestmark = pytest.mark.gpu


def _batch(seed, n, L_range, r_range):
    shapes = inputs.batch_shapes(seed, n, L_range, r_range)
    xs, ws = [], []
    for i, (L, r, a) in enumerate(shapes):
        xs.append(inputs.random_tt(seed * 1000 + i, L, 2, r))
        ws.append(inputs.random_mpo(seed * 1000 + 500 + i, L, 2, a))
    return xs, ws


@pytest.mark.parametrize("nstreams", [1, 4])
def test_batched_fp64_small(cuda_lib, nstreams):
    tt = cuda_lib
    xs, ws = _batch(7, 12, (3, 10), (2, 9))
    X = [tt.TT.from_numpy(x) for x in xs]
    W = [tt.MPO.from_numpy(w) for w in ws]
    outs = tt.tt_apply_round_batched(W, X, 1e-10, nstreams=nstreams)
    for x, w, o in zip(xs, ws, outs):
        ref = core.round_tt(core.apply_mpo(w, x), 1e-10)
        got = o.numpy()
        assert core.ranks(got) == core.ranks(ref)
        assert core.rel_err(got, ref) <= 1e-12


def test_batched_mixed_uneven(cuda_lib):
    """Trains with L in [20, 60] and ranks in [8, 40], FP32 cores, eps = 1e-6."""
    tt = cuda_lib
    xs, ws = _batch(8, 6, (20, 60), (8, 40))
    xs = [[c.astype(np.float32) for c in x] for x in xs]
    ws = [[c.astype(np.float32) for c in w] for w in ws]
    X = [tt.TT.from_numpy(x, dtype=torch.float32) for x in xs]
    W = [tt.MPO.from_numpy(w, dtype=torch.float32) for w in ws]
    outs = tt.tt_apply_round_batched(W, X, 1e-6, nstreams=3)
    for x, w, o in zip(xs, ws, outs):
        y = core.apply_mpo([c.astype(np.float64) for c in w], [c.astype(np.float64) for c in x])
        ref = core.round_tt(y, 1e-6)
        e = core.rel_err(o.numpy(), ref)
        assert e <= 4e-6, e


def _custom_batch():
    """Lengths 4..9 in one batch, wide bonds (rank 40 next to d r_0 = 2), heavy truncation."""
    spec = [(6, [1, 40, 40, 40, 40, 40, 1], 2), (9, 6, 3), (4, 3, 2), (7, [1, 2, 4, 30, 30, 4, 2, 1], 3),
            (5, 12, 1)]
    xs, ws = [], []
    for i, (L, r, a) in enumerate(spec):
        xs.append(inputs.random_tt(300 + i, L, 2, r))
        ws.append(inputs.random_mpo(350 + i, L, 2, a))
    return xs, ws


@pytest.mark.parametrize("eps", [1e-3, 1e-9])
def test_batched_fp64_ragged_truncating(cuda_lib, eps):
    tt = cuda_lib
    xs, ws = _custom_batch()
    X = [tt.TT.from_numpy(x) for x in xs]
    W = [tt.MPO.from_numpy(w) for w in ws]
    outs = tt.tt_apply_round_batched(W, X, eps)
    for x, w, o in zip(xs, ws, outs):
        ref = core.round_tt(core.apply_mpo(w, x), eps)
        got = o.numpy()
        assert core.ranks(got) == core.ranks(ref)
        assert core.rel_err(got, ref) <= 1e-12


def test_batched_mixed_ragged(cuda_lib):
    tt = cuda_lib
    xs, ws = _custom_batch()
    xs = [[c.astype(np.float32) for c in x] for x in xs]
    ws = [[c.astype(np.float32) for c in w] for w in ws]
    X = [tt.TT.from_numpy(x, dtype=torch.float32) for x in xs]
    W = [tt.MPO.from_numpy(w, dtype=torch.float32) for w in ws]
    outs = tt.tt_apply_round_batched(W, X, 1e-6)
    for x, w, o in zip(xs, ws, outs):
        y = core.apply_mpo([c.astype(np.float64) for c in w], [c.astype(np.float64) for c in x])
        assert core.rel_err(o.numpy(), core.round_tt(y, 1e-6)) <= 2e-6
