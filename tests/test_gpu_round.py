"""GPU parity of TT rounding (FP64 form) against the oracle.

SVD factors are not unique, so the comparison is gauge-invariant:
e(a, b) = ||a - b|| / ||b|| through the exact block sum (oracle), plus equal ranks,
left-orthonormal output cores and the rounding bound.  Bar: e <= 1e-12 for the FP64
form (the tolerance the paper's hot path is held to).
"""
import math

import numpy as np
import pytest
import torch

from oracle import core, structured
from paper_2602_20226_gb300 import inputs, qtt

pytestmark = pytest.mark.gpu


def _round_gpu(tt, x_np, eps, max_rank=0):
    X = tt.TT.from_numpy(x_np, dtype=torch.float64)
    Y, nrm = tt.tt_round(X, eps, max_rank)
    return Y.numpy(), nrm


def _check(y_gpu, y_ref, x, eps, tol=1e-12):
    assert core.ranks(y_gpu) == core.ranks(y_ref)
    assert core.rel_err(y_gpu, y_ref) <= tol
    for k in range(len(y_gpu) - 1):
        assert core.left_orthogonality_defect(y_gpu[k]) <= 1e-12
    # rounding bound against the input
    assert core.rel_err(y_gpu, x) <= eps * (1 + 1e-6) + 1e-13


def test_round_c1_second_difference(cuda_lib):
    """L = 10, r = 8, 1D Dirichlet second difference (rank 3), eps = 1e-10."""
    x = inputs.random_tt(1, 10, 2, 8)
    y = core.apply_mpo(structured.laplacian_mpo(1, 10), x)
    ref, info = core.round_tt(y, 1e-10, return_info=True)
    got, nrm = _round_gpu(cuda_lib, y, 1e-10)
    assert abs(nrm - info["norm"]) <= 1e-13 * info["norm"]
    _check(got, ref, y, 1e-10)


def test_round_c1_sin_closed_form(cuda_lib):
    """round(Delta sin(2 pi x)) = lambda sin(2 pi x) with rank 2, on the GPU."""
    bits = 10
    N = 2 ** bits
    lo, hi = 1.0 / (N + 1), N / (N + 1.0)
    tt = cuda_lib
    v = qtt.sin_tt(bits, lo, hi, 2 * math.pi)
    W = tt.MPO.from_numpy(qtt.second_difference_mpo(bits))
    Y = tt.tt_apply_mpo(W, tt.TT.from_numpy(v))
    Z, _ = tt.tt_round(Y, 1e-10)
    assert Z.ranks == [1] + [2] * (bits - 1) + [1]
    lam = -4 * math.sin(math.pi / (N + 1)) ** 2
    ref = structured.sin_tt([2] * bits, lo, hi, 2 * math.pi)
    # Delta v cancels O(1) terms down to O(|lambda|): attainable error ~ 4u/|lambda|
    assert core.rel_err(Z.numpy(), core.scale(ref, lam)) <= max(1e-12, 50 * 2.2e-16 / abs(lam))


def test_round_c2_laplacian_full_size(cuda_lib):
    """L = 40 (2 x 20 interleaved), r = 64, 2D Laplacian (rank 5) -> n = 320, eps = 1e-8."""
    tt = cuda_lib
    x = inputs.random_tt(2, 40, 2, 64)
    W = qtt.laplacian_mpo(2, 20)
    Y = tt.tt_apply_mpo(tt.MPO.from_numpy(W), tt.TT.from_numpy(x))
    y = core.apply_mpo(structured.laplacian_mpo(2, 20), x)
    assert Y.ranks == core.ranks(y)
    Z, nrm = tt.tt_round(Y, 1e-8)
    ref, info = core.round_tt(y, 1e-8, return_info=True)
    assert abs(nrm - info["norm"]) <= 1e-13 * info["norm"]
    got = Z.numpy()
    assert core.ranks(got) == info["ranks"]
    assert core.rel_err(got, ref) <= 1e-12
    for k in range(0, 39, 6):
        assert core.left_orthogonality_defect(got[k]) <= 1e-12


@pytest.mark.parametrize("case", ["modes", "odd_ranks", "two_sites", "one_site", "wide_left"])
def test_round_ragged(cuda_lib, case):
    eps = 1e-6
    if case == "modes":
        x = inputs.random_tt(3, 6, [2, 3, 5, 2, 3, 2], [1, 6, 7, 9, 5, 4, 1])
    elif case == "odd_ranks":
        x = core.add(inputs.random_tt(4, 9, 2, [1, 2, 5, 13, 31, 33, 17, 7, 3, 1]),
                     core.scale(inputs.random_tt(5, 9, 2, 3), 1e-4))
        eps = 1e-3
    elif case == "two_sites":
        x = inputs.random_tt(6, 2, 16, [1, 16, 1])
    elif case == "one_site":
        x = inputs.random_tt(7, 1, 9, [1, 1])
    else:
        x = inputs.random_tt(8, 5, 2, [1, 40, 40, 40, 40, 1])
    ref = core.round_tt(x, eps)
    got, _ = _round_gpu(cuda_lib, x, eps)
    _check(got, ref, x, eps)


def test_round_redundant_ranks_and_cap(cuda_lib):
    L, r = 12, 8
    x = inputs.random_tt(9, L, 2, r)
    got, _ = _round_gpu(cuda_lib, x, 1e-14)
    assert core.ranks(got) == [1] + [min(r, 2 ** k, 2 ** (L - k)) for k in range(1, L)] + [1]
    assert core.rel_err(got, x) <= 1e-13
    capped, _ = _round_gpu(cuda_lib, x, 1e-14, max_rank=3)
    ref = core.round_tt(x, 1e-14, max_rank=3)
    assert max(core.ranks(capped)) == 3
    assert core.rel_err(capped, ref) <= 1e-12


def test_round_zero_tensor(cuda_lib):
    x = core.scale(inputs.random_tt(10, 6, 2, 3), 0.0)
    got, nrm = _round_gpu(cuda_lib, x, 1e-8)
    assert nrm == 0.0
    assert core.ranks(got) == [1] * 7
    assert all(np.all(c == 0.0) for c in [got[-1]])
    assert np.all(core.full(got) == 0.0)


def test_round_hadamard_square(cuda_lib):
    """x (.) x then round: interior ranks <= r(r+1)/2 (symmetric subspace)."""
    tt = cuda_lib
    L, r = 14, 6
    x = inputs.random_tt(11, L, 2, r)
    X = tt.TT.from_numpy(x)
    Z, _ = tt.tt_round(tt.tt_hadamard(X, X), 1e-10)
    ref = core.round_tt(core.hadamard(x, x), 1e-10)
    got = Z.numpy()
    assert core.ranks(got) == core.ranks(ref)
    assert max(core.ranks(got)) <= r * (r + 1) // 2
    assert core.rel_err(got, ref) <= 1e-12


def test_round_is_deterministic(cuda_lib):
    x = inputs.random_tt(12, 10, 2, 24)
    a, _ = _round_gpu(cuda_lib, x, 1e-6)
    b, _ = _round_gpu(cuda_lib, x, 1e-6)
    assert all(np.array_equal(u, v) for u, v in zip(a, b))
