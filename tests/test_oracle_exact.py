"""Pins for the oracle's exact operations (Sections 2 and 3.1) against brute force.

Every check compares the TT-level routine with the same quantity computed on the
full tensor (dense numpy arrays), which shares nothing with the core-by-core code.
"""
import numpy as np
import pytest

from oracle import core, structured
from paper_2602_20226_gb300 import inputs


def _rand_tt(seed, d, r):
    L = len(d)
    ranks = [1] + [r] * (L - 1) + [1]
    return inputs.random_tt(seed, L, d, ranks)


def _rand_mpo(seed, d, a):
    g = inputs.rng(seed)
    L = len(d)
    ranks = [1] + [a] * (L - 1) + [1]
    return [g.standard_normal((ranks[k], d[k], d[k], ranks[k + 1])) for k in range(L)]


@pytest.mark.parametrize("d", [[2] * 8, [2, 3, 5, 2, 3]])
def test_full_matches_explicit_products(d):
    x = _rand_tt(1, d, 3)
    t = core.full(x)
    rng = np.random.default_rng(0)
    for _ in range(20):
        idx = tuple(int(rng.integers(0, b)) for b in d)
        v = np.ones((1, 1))
        for k, i in enumerate(idx):
            v = v @ x[k][:, i, :]
        assert abs(t[idx] - v[0, 0]) <= 1e-14 * max(1.0, abs(v[0, 0]))


@pytest.mark.parametrize("d", [[2] * 8, [2, 3, 5, 2]])
def test_apply_mpo_is_matvec(d):
    x = _rand_tt(2, d, 4)
    w = _rand_mpo(3, d, 3)
    y = core.apply_mpo(w, x)
    assert core.ranks(y) == [1] + [12] * (len(d) - 1) + [1]
    lhs = core.full(y).reshape(-1)
    rhs = core.full_mpo(w) @ core.full(x).reshape(-1)
    assert np.allclose(lhs, rhs, rtol=1e-12, atol=1e-12 * np.abs(rhs).max())


def test_apply_mpo_bond_flatten_operator_major():
    """xi = a * R_x + r: an operator block in bond a lands in rows a*R_x .. a*R_x + R_x - 1."""
    d = [2, 2, 2]
    x = _rand_tt(4, d, 3)
    w = _rand_mpo(5, d, 2)
    # keep only the (a=1 -> a'=0) block of the middle operator core
    w[1] = np.zeros_like(w[1])
    w[1][1, :, :, 0] = np.array([[1.0, 2.0], [3.0, 4.0]])
    y = core.apply_mpo(w, x)
    rx = 3
    mid = y[1]
    assert np.all(mid[:rx] == 0.0)          # rows of operator bond 0 are empty
    assert np.all(mid[:, :, rx:] == 0.0)    # columns of operator bond 1 are empty
    blk = mid[rx:2 * rx, :, :rx]            # (a=1, r) x i x (a'=0, r')
    want = np.einsum("ij,rjs->ris", w[1][1, :, :, 0], x[1])
    assert np.array_equal(blk, want)


@pytest.mark.parametrize("d", [[2] * 9, [3, 2, 5, 2]])
def test_hadamard_is_elementwise(d):
    x = _rand_tt(6, d, 3)
    y = _rand_tt(7, d, 2)
    z = core.hadamard(x, y)
    assert core.ranks(z) == [1] + [6] * (len(d) - 1) + [1]
    assert np.allclose(core.full(z), core.full(x) * core.full(y), rtol=1e-12, atol=1e-14)


def test_hadamard_flatten_first_operand_major():
    d = [2, 2, 2]
    x = _rand_tt(8, d, 2)
    y = _rand_tt(9, d, 3)
    z = core.hadamard(x, y)
    # Z_1[(r,s), i, (r',s')] = X[r,i,r'] Y[s,i,s'], index r*3+s
    for r in range(2):
        for s in range(3):
            for rp in range(2):
                for sp in range(3):
                    assert z[1][r * 3 + s, 1, rp * 3 + sp] == x[1][r, 1, rp] * y[1][s, 1, sp]


@pytest.mark.parametrize("d", [[2] * 7, [2, 5, 3]])
def test_add_block_sum(d):
    x = _rand_tt(10, d, 3)
    y = _rand_tt(11, d, 4)
    s = core.add(x, y)
    assert core.ranks(s) == [1] + [7] * (len(d) - 1) + [1]
    assert np.allclose(core.full(s), core.full(x) + core.full(y), rtol=1e-12, atol=1e-14)


def test_inner_and_norm_brute_force():
    d = [2] * 10
    x = _rand_tt(12, d, 5)
    y = _rand_tt(13, d, 4)
    fx, fy = core.full(x), core.full(y)
    assert abs(core.inner(x, y) - np.sum(fx * fy)) <= 1e-13 * np.linalg.norm(fx) * np.linalg.norm(fy)
    assert abs(core.norm(x) - np.linalg.norm(fx)) <= 1e-13 * np.linalg.norm(fx)


def test_inner_closed_form_exponentials():
    """<e^{alpha x}, e^{beta x}> is a geometric series in e^{(alpha+beta) h}."""
    bits = 12
    bases = [2] * bits
    a, b = -1.0, 1.0
    alpha, beta = 0.7, -1.9
    ea = structured.exp_tt(bases, a, b, alpha)
    eb = structured.exp_tt(bases, a, b, beta)
    n = 2 ** bits
    h = (b - a) / (n - 1)
    q = np.exp((alpha + beta) * h)
    want = np.exp((alpha + beta) * a) * (1 - q ** n) / (1 - q)
    assert abs(core.inner(ea, eb) - want) <= 1e-12 * abs(want)


@pytest.mark.parametrize("d", [[2] * 10, [2, 3, 5, 2, 7]])
def test_evaluate_brute_force(d):
    x = _rand_tt(14, d, 6)
    digs = inputs.random_digits(15, 300, d)
    v = core.evaluate(x, digs)
    t = core.full(x)
    want = t[tuple(digs[:, k].astype(np.int64) for k in range(len(d)))]
    assert np.allclose(v, want, rtol=1e-12, atol=1e-15)


def test_rel_err_brute_force():
    d = [2] * 9
    x = _rand_tt(16, d, 4)
    y = _rand_tt(17, d, 3)
    e = core.rel_err(x, y)
    fx, fy = core.full(x), core.full(y)
    assert abs(e - np.linalg.norm(fx - fy) / np.linalg.norm(fy)) <= 1e-12
    assert core.rel_err(x, x) <= 1e-14
    assert abs(core.rel_err(core.scale(x, 2.0), x) - 1.0) <= 1e-13


def test_quantization_digits_roundtrip():
    bases = [2, 5, 2]  # the explicit factorisation 2*5*2 of 20
    idx = np.arange(20)
    dg = structured.to_digits(idx, bases)
    assert np.array_equal(structured.to_idxs(dg, bases), idx)
    # most significant digit first: c = (10, 2, 1)
    assert structured.coefficients(bases) == [10, 2, 1]
    assert dg[13].tolist() == [1, 1, 1]
