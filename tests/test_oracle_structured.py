"""Pins for the oracle's structured tensors (Section 4) against dense definitions."""
import math
import os

import numpy as np
import pytest

from oracle import core, structured

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("bases", [[2] * 10, [2, 3, 5, 2, 3], [7, 2, 2, 3]])
def test_exp_closed_form(bases):
    a, b, v, x0 = -1.0, 2.0, 1.3, 0.25
    t = structured.exp_tt(bases, a, b, v, x0)
    assert core.ranks(t) == [1] * (len(bases) + 1)
    x = structured.grid_points(bases, a, b)
    assert np.allclose(core.full(t).reshape(-1), np.exp(v * (x - x0)), rtol=1e-13, atol=0)


@pytest.mark.parametrize("bases", [[2] * 12, [2, 3, 5, 2, 3]])
def test_cos_sin_closed_form(bases):
    a, b, v, x0 = -1.0, 1.0, 7.0, 0.1
    x = structured.grid_points(bases, a, b)
    c = structured.cos_tt(bases, a, b, v, x0)
    s = structured.sin_tt(bases, a, b, v, x0)
    assert max(core.ranks(c)) == 2 and max(core.ranks(s)) == 2
    L = len(bases)
    assert np.max(np.abs(core.full(c).reshape(-1) - np.cos(v * (x - x0)))) <= 1e-14 * L * 4
    assert np.max(np.abs(core.full(s).reshape(-1) - np.sin(v * (x - x0)))) <= 1e-14 * L * 4


@pytest.mark.parametrize("coeffs", [[1.0, 0.0, 0.1], [0.3, -1.0, 0.5, 2.0, -0.7]])
def test_polynomial_closed_form(coeffs):
    bases = [2, 3, 2, 5, 2]
    a, b, x0 = -1.0, 1.0, 0.5
    t = structured.poly_tt(bases, a, b, coeffs, x0)
    p = len(coeffs) - 1
    assert max(core.ranks(t)) == p + 1
    x = structured.grid_points(bases, a, b)
    want = sum(c * (x - x0) ** s for s, c in enumerate(coeffs))
    assert np.allclose(core.full(t).reshape(-1), want, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("bases,shift", [([2] * 6, 1), ([2] * 6, 13), ([2, 3, 5], 7), ([3, 2, 2, 2], 0),
                                         ([2, 5, 2], 19)])
def test_shift_mpo_is_shift_matrix(bases, shift):
    w = structured.shift_mpo(bases, shift)
    assert max(core.ranks(w)) <= 2
    n = int(np.prod(bases))
    assert np.array_equal(core.full_mpo(w), np.eye(n, k=-shift))


def test_shift_cores_golden():
    """Base-2 cores of Q_1 (Eq. (shif_dec)) against the hand-written fixture."""
    want = {}
    with open(os.path.join(GOLDEN, "shift_b2_cores.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            name, vals = line.split(":")
            want[name.strip()] = np.array([float(v) for v in vals.split()]).reshape(2, 2)
    w = structured.shift_mpo([2] * 4, 1)
    mid = w[1]
    assert np.array_equal(mid[0, :, :, 0], want["Q0"])
    assert np.array_equal(mid[0, :, :, 1], want["Q1"])
    assert np.array_equal(mid[1, :, :, 0], want["R0"])
    assert np.array_equal(mid[1, :, :, 1], want["R1"])
    assert np.array_equal(w[-1][0, :, :, 0], want["Q1"])
    assert np.array_equal(w[-1][1, :, :, 0], want["R1"])


@pytest.mark.parametrize("n_dims,bits,rank", [(1, 8, 3), (2, 4, 5), (3, 3, 7)])
def test_laplacian_dense(n_dims, bits, rank):
    w = structured.laplacian_mpo(n_dims, bits)
    assert max(core.ranks(w)) == rank
    dense = core.full_mpo(w)
    perm = structured.interleaved_permutation(n_dims, bits)
    want = structured.dense_laplacian(n_dims, bits)
    # dense is in interleaved flat order; permute to natural order
    nat = np.empty_like(dense)
    nat[np.ix_(perm, perm)] = dense
    assert np.array_equal(nat, want)
    # and equal to the (non-minimal) exact sum of shifted identities
    assert np.array_equal(core.full_mpo(structured.laplacian_mpo_sum(n_dims, bits)), dense)


def test_laplacian_2d_bond_ranks():
    """Interleaved 2D: bond 1 has rank 3, the bond between the last x and y digit rank 4."""
    w = structured.laplacian_mpo(2, 5)
    rk = core.ranks(w)
    assert rk[0] == 1 and rk[-1] == 1
    assert rk[1] == 3
    assert rk[-2] == 4
    assert max(rk) == 5


def test_second_difference_small_dense():
    w = structured.laplacian_mpo(1, 3)
    want = -2 * np.eye(8) + np.eye(8, k=1) + np.eye(8, k=-1)
    assert np.array_equal(core.full_mpo(w), want)


def test_laplacian_on_sin_eigenvalue_pointwise():
    bits = 9
    N = 2 ** bits
    lo, hi = 1.0 / (N + 1), N / (N + 1.0)
    v = structured.sin_tt([2] * bits, lo, hi, 2 * math.pi)
    y = core.apply_mpo(structured.laplacian_mpo(1, bits), v)
    lam = -4 * math.sin(math.pi / (N + 1)) ** 2
    assert np.allclose(core.full(y).reshape(-1), lam * core.full(v).reshape(-1), atol=1e-13)
