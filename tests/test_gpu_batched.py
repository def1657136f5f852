"""Batched apply + round over trains of uneven length and rank (tt_apply_round_batched).

Every train of the batch is checked against the oracle's apply + round on the same
seeded inputs: FP64 form e <= 1e-12 with equal ranks; mixed form (FP32 cores) e <= 1e-6
at eps = 1e-6 with equal ranks, on short ragged batches, on 20..60-site trains and on
trains at the top of the uneven batch's range (rank 96..128, MPO rank 4..5, bonds up to
640, which run the largest cluster sizes of the batched bond SVDs).  The mixed form's QR
factors each panel in FP64 (reflectors rounded to FP32, T recomputed from them) and keeps
the block-reflector products in FP64; the remaining error is the FP32 storage of the cores
between the sweep steps (a CPU emulation of the chain puts it at 5e-7..8e-7 on these
trains).
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
        got = o.numpy()
        assert core.ranks(got) == core.ranks(ref)
        e = core.rel_err(got, ref)
        assert e <= 1e-6, e


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
        ref = core.round_tt(y, 1e-6)
        got = o.numpy()
        assert core.ranks(got) == core.ranks(ref)
        assert core.rel_err(got, ref) <= 1e-6


def _e_from_inner(a, b):
    """e(a, b) from the oracle's FP64 inner products: (|a|^2 + |b|^2 - 2 <a, b>)^(1/2) / |b|.
    The cancellation limits its resolution to about 2e-7 (FP64 environments of ~50 sites),
    enough for the mixed form's 1e-6 and far cheaper than the block-sum QR of rel_err on
    bonds of 640 (a rank-1280 sweep)."""
    aa, bb, ab = core.inner(a, a), core.inner(b, b), core.inner(a, b)
    return float(np.sqrt(max(aa + bb - 2.0 * ab, 0.0) / bb))


def _sampled_entries(a, b, seed, n=2048):
    """Largest difference of n sampled entries, relative to the RMS of b's sampled entries."""
    dg = inputs.random_digits(seed, n, [c.shape[1] for c in b])
    va, vb = core.evaluate(a, dg), core.evaluate(b, dg)
    return float(np.abs(va - vb).max() / np.sqrt(np.mean(vb * vb)))


def test_batched_full_size_both_forms(cuda_lib):
    """Trains at the top of the uneven batch's range, in both forms on the same FP32 values:
    FP64 with equal ranks and sampled entries within 1e-11 of the RMS entry (the exact
    block-sum metric, a rank-1280 sweep per train, is left to the single-train tests at
    bond 320), mixed e <= 1e-6 with equal ranks."""
    tt = cuda_lib
    spec = [(44, 96, 5), (40, 128, 5), (56, 120, 4)]
    xs = [[c.astype(np.float32) for c in inputs.random_tt(6100 + i, L, 2, r)] for i, (L, r, a) in enumerate(spec)]
    ws = [[c.astype(np.float32) for c in inputs.random_mpo(6200 + i, L, 2, a)] for i, (L, r, a) in enumerate(spec)]
    refs = []
    for x, w in zip(xs, ws):
        y = core.apply_mpo([c.astype(np.float64) for c in w], [c.astype(np.float64) for c in x])
        refs.append(core.round_tt(y, 1e-6))
    for dt in (torch.float64, torch.float32):
        X = [tt.TT.from_numpy(x, dtype=dt) for x in xs]
        W = [tt.MPO.from_numpy(w, dtype=dt) for w in ws]
        outs = tt.tt_apply_round_batched(W, X, 1e-6)
        for i, (o, ref) in enumerate(zip(outs, refs)):
            got = o.numpy()
            assert core.ranks(got) == core.ranks(ref), (i, dt)
            if dt == torch.float64:
                assert _sampled_entries(got, ref, 6300 + i) <= 1e-11
            else:
                e = _e_from_inner(got, ref)
                assert e <= 1e-6, (i, e)
                assert _sampled_entries(got, ref, 6300 + i) <= 2e-5
