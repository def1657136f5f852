"""Pins for the oracle's orthogonalisation and rounding (Section 3.2).

Checks against: the full tensor (brute force), orthonormality of the swept cores,
the rounding bound ||x - round(x)|| <= eps ||x||, the Eckart-Young optimum for
L = 2 (truncated SVD of the full matrix), exact ranks of redundant TTs and the
closed-form ranks of Section 4.1.
"""
import math

import numpy as np
import pytest

from oracle import core, structured
from paper_2602_20226_gb300 import inputs


def _tt(seed, L, r, d=2):
    return inputs.random_tt(seed, L, d, r)


def test_orthogonalize_keeps_tensor_and_orthonormalises():
    x = _tt(1, 10, 6)
    c = core.orthogonalize_rl(x)
    assert np.allclose(core.full(c), core.full(x), rtol=1e-12, atol=1e-14)
    for k in range(1, len(c)):
        assert core.right_orthogonality_defect(c[k]) <= 1e-13
    # ranks after the sweep never exceed min(r, d^(L-k))
    rk = core.ranks(c)
    for k in range(1, 10):
        assert rk[k] <= min(6, 2 ** (10 - k))


def test_norm_from_first_core():
    x = _tt(2, 11, 5)
    assert abs(core.norm(x) - np.linalg.norm(core.full(x))) <= 1e-13 * np.linalg.norm(core.full(x))


def test_round_redundant_ranks_exact():
    """With eps ~ machine precision, ranks drop to min(r, d^k, d^(L-k)) and nothing else changes."""
    L, r = 12, 8
    x = _tt(3, L, r)
    y, info = core.round_tt(x, 1e-14, return_info=True)
    want = [1] + [min(r, 2 ** k, 2 ** (L - k)) for k in range(1, L)] + [1]
    assert info["ranks"] == want
    assert np.linalg.norm(core.full(y) - core.full(x)) <= 1e-13 * np.linalg.norm(core.full(x))
    for k in range(L - 1):
        assert core.left_orthogonality_defect(y[k]) <= 1e-13


@pytest.mark.parametrize("eps", [1e-1, 3e-2, 1e-2])
def test_rounding_bound(eps):
    L = 12
    x = core.add(_tt(4, L, 6), core.scale(_tt(5, L, 3), 1e-2))
    y = core.round_tt(x, eps)
    fx = core.full(x)
    err = np.linalg.norm(core.full(y) - fx)
    assert err <= eps * np.linalg.norm(fx) * (1 + 1e-12)
    assert max(core.ranks(y)) < max(core.ranks(x))


def test_round_two_sites_is_truncated_svd():
    """For L = 2 rounding is the truncated SVD of the 2-site matrix (Eckart-Young)."""
    g = np.random.default_rng(7)
    m = g.standard_normal((16, 16)) @ np.diag(np.logspace(0, -6, 16)) @ g.standard_normal((16, 16))
    x = [m.reshape(1, 16, 16), np.eye(16).reshape(16, 16, 1)]
    nrm = np.linalg.norm(m)
    s = np.linalg.svd(m, compute_uv=False)
    for eps in [1e-2, 1e-4]:
        y = core.round_tt(x, eps)
        delta = eps * nrm  # sqrt(L - 1) = 1
        tails = np.sqrt(np.cumsum((s ** 2)[::-1]))[::-1]  # tails[j] = ||s[j:]||
        r_want = next(j for j in range(1, 17) if j == 16 or tails[j] <= delta)
        assert core.ranks(y)[1] == r_want
        err = np.linalg.norm(core.full(y).reshape(16, 16) - m)
        assert abs(err - (tails[r_want] if r_want < 16 else 0.0)) <= 1e-12 * nrm


def _orthogonal_terms_tt(s, L, d, seed):
    """x = sum_j s_j a_j^(1) (x) ... (x) a_j^(L), the a_j^(k) orthonormal over j at every site.

    Every unfolding of x is then sum_j s_j (left_j)(right_j)^T with orthonormal left and right
    factors, so its singular values are exactly s, at every bond."""
    m = len(s)
    g = np.random.default_rng(seed)
    vecs = [np.linalg.qr(g.standard_normal((d, m)))[0] for _ in range(L)]  # d x m, orthonormal columns
    cores = [np.einsum("ij,j->ij", vecs[0], s).reshape(1, d, m)]
    for k in range(1, L - 1):
        c = np.zeros((m, d, m))
        for j in range(m):
            c[j, :, j] = vecs[k][:, j]
        cores.append(c)
    cores.append(vecs[L - 1].T.reshape(m, d, 1))
    # an invertible gauge G_k at every bond (core k <- core k G_k, core k+1 <- G_k^-1 core k+1):
    # the tensor is unchanged, but the cores are no longer orthogonal and the first one carries
    # 3 ||x|| (G_1 = 3 x an orthogonal matrix)
    for k in range(L - 1):
        if k == 0:
            gk = 3.0 * np.linalg.qr(g.standard_normal((m, m)))[0]
        else:
            gk = np.eye(m) + 0.3 * g.standard_normal((m, m))
        cores[k] = np.einsum("adb,bc->adc", cores[k], gk)
        cores[k + 1] = np.einsum("ab,bdc->adc", np.linalg.inv(gk), cores[k + 1])
    return cores


@pytest.mark.parametrize("L", [3, 5, 9])
def test_round_known_bond_spectrum(L):
    """Bond spectrum s at every bond (above): round_tt keeps, at every bond, the smallest r'
    whose tail (sum_{j >= r'} s_j^2)^(1/2) is <= delta = eps ||x|| / sqrt(L - 1), and its error is
    exactly that tail (the dropped terms are orthogonal to the kept ones).  eps is set so that
    delta sits at 0.7x and 1.4x of each tail, so a threshold off by sqrt(L - 1) >= 2 (L >= 5), a
    norm read off the gauged input instead of the orthogonalised first core (3x), or a misplaced
    tail moves the rank."""
    s = np.array([1.0, 0.5, 0.1, 0.02])
    x = _orthogonal_terms_tt(s, L, 5, seed=40 + L)
    fx = core.full(x)
    nrm = float(np.linalg.norm(s))
    assert abs(np.linalg.norm(fx) - nrm) <= 1e-13
    assert abs(np.linalg.norm(x[0]) - 3.0 * nrm) <= 1e-13  # the input's first core is not the norm
    tails = [float(np.sqrt(np.sum(s[j:] ** 2))) for j in range(len(s) + 1)]  # tails[4] = 0
    for t in (1, 2, 3):
        for factor in (0.7, 1.4):
            delta = factor * tails[t]
            eps = delta * math.sqrt(L - 1) / nrm
            y = core.round_tt(x, eps)
            r_want = min(j for j in range(1, len(s) + 1) if tails[j] <= delta)
            assert r_want == (t if factor > 1 else t + 1)
            assert core.ranks(y) == [1] + [r_want] * (L - 1) + [1], (t, factor)
            err = np.linalg.norm(core.full(y) - fx)
            assert abs(err - tails[r_want]) <= 1e-13, (t, factor, err)


def test_round_max_rank_cap():
    x = _tt(8, 10, 6)
    y = core.round_tt(x, 1e-14, max_rank=3)
    assert max(core.ranks(y)) == 3


def test_truncation_rank_rule():
    s = np.array([4.0, 2.0, 1.0, 0.5])
    assert core.truncation_rank(s, 0.0) == 4
    assert core.truncation_rank(s, 0.5) == 3           # tail {0.5} = 0.5 <= 0.5 (inclusive)
    assert core.truncation_rank(s, math.sqrt(1.25)) == 2
    assert core.truncation_rank(s, 100.0) == 1          # never below rank 1
    assert core.truncation_rank(np.zeros(5), 0.0) == 1  # zero tensor -> rank 1


def test_round_zero_tensor():
    x = core.scale(_tt(9, 6, 3), 0.0)
    y = core.round_tt(x, 1e-8)
    assert core.ranks(y) == [1] * 7
    assert np.all(core.full(y) == 0.0)


def test_round_closed_form_ranks():
    bases = [2] * 14
    e1 = structured.exp_tt(bases, -1.0, 1.0, 0.8)
    e2 = structured.exp_tt(bases, -1.0, 1.0, -2.5)
    s = core.add(core.add(e1, e2), e1)  # rank 3 representation of a rank-2 function
    y = core.round_tt(s, 1e-12)
    assert max(core.ranks(y)) == 2
    sn = structured.sin_tt(bases, -1.0, 1.0, 3.0)
    sq = core.round_tt(core.hadamard(sn, sn), 1e-12)  # sin^2 = (1 - cos 2t)/2 -> rank 3
    assert max(core.ranks(sq)) == 3
    ee = core.round_tt(core.hadamard(e1, e1), 1e-12)
    assert max(core.ranks(ee)) == 1
    p = structured.poly_tt(bases, -1.0, 1.0, [0.3, -1.0, 0.0, 2.0])  # degree 3
    pr = core.round_tt(core.add(p, p), 1e-12)
    assert max(core.ranks(pr)) <= 4


def test_hadamard_square_symmetric_rank():
    """x (.) x lives in the symmetric part of the bond space: rank <= r(r+1)/2."""
    L, r = 12, 3
    x = _tt(10, L, r)
    z = core.round_tt(core.hadamard(x, x), 1e-12)
    for k in range(1, L):
        assert core.ranks(z)[k] <= min(r * (r + 1) // 2, 2 ** k, 2 ** (L - k))


@pytest.mark.parametrize("n_dims,bits", [(1, 6), (2, 4), (3, 3)])
def test_dirichlet_eigenvector(n_dims, bits):
    """sin(2 pi x) on x_i = (i+1)/(N+1) is an eigenvector of the Dirichlet Laplacian.

    round(Delta v) must have the rank of v (2 per dimension factor) and equal lambda v,
    lambda = -4 sin^2(pi/(N+1)) per dimension.  Delta v cancels three O(1) terms down
    to O(|lambda|), so the attainable relative error is about 4 n_dims u / |lambda|;
    the grids are small enough that this stays far below the 1e-12 bar.
    """
    N = 2 ** bits
    lo, hi = 1.0 / (N + 1), N / (N + 1.0)
    one = structured.sin_tt([2] * bits, lo, hi, 2 * math.pi)
    # v = prod_t sin(2 pi x_t) on the interleaved layout
    L = n_dims * bits
    v = None
    layout = structured.interleaved_layout(n_dims, bits)
    for t in range(n_dims):
        cores, it, cur = [], iter(one), 1
        for k in range(L):
            if layout[k] == t:
                c = next(it)
                cur = c.shape[-1]
                cores.append(c)
            else:
                cores.append(np.stack([np.eye(cur)] * 2, axis=1))
        v = cores if v is None else core.hadamard(v, cores)
    v = core.round_tt(v, 1e-14)
    lam = -4.0 * math.sin(math.pi / (N + 1)) ** 2 * n_dims
    w = structured.laplacian_mpo(n_dims, bits)
    y = core.round_tt(core.apply_mpo(w, v), 1e-10)
    assert max(core.ranks(y)) == 2 ** n_dims
    assert 4 * n_dims * 2.2e-16 / abs(lam) < 1e-13
    assert core.rel_err(y, core.scale(v, lam)) <= 1e-12
