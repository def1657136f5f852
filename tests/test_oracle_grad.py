"""Pins for the oracle's hand-derived adjoints against FP64 central finite differences.

For a scalar loss l(theta), each core entry theta is perturbed by
h = 1e-6 max(1, |theta|); (l(theta+h) - l(theta-h)) / 2h must match the adjoint to
1e-7 relative (the O(h^2) truncation plus rounding of the difference quotient).
"""
import numpy as np
import pytest

from oracle import core, grad
from paper_2602_20226_gb300 import inputs


def _fd_check(loss, params, grads, n_probe=25, seed=0):
    rng = np.random.default_rng(seed)
    scale = max(np.abs(g).max() for g in grads) + 1e-300
    for _ in range(n_probe):
        k = int(rng.integers(0, len(params)))
        idx = tuple(int(rng.integers(0, s)) for s in params[k].shape)
        th = params[k][idx]
        h = 1e-6 * max(1.0, abs(th))
        params[k][idx] = th + h
        lp = loss()
        params[k][idx] = th - h
        lm = loss()
        params[k][idx] = th
        fd = (lp - lm) / (2 * h)
        assert abs(fd - grads[k][idx]) <= 1e-7 * scale, (k, idx, fd, grads[k][idx])


def _tt(seed, L, r, d=2):
    return inputs.random_tt(seed, L, d, r)


def test_inner_vjp_fd():
    x = _tt(1, 7, 4)
    y = _tt(2, 7, 3)
    dx, dy = grad.inner_vjp(x, y, 1.7)
    _fd_check(lambda: 1.7 * core.inner(x, y), x, dx)
    _fd_check(lambda: 1.7 * core.inner(x, y), y, dy, seed=1)


def test_apply_vjp_fd():
    x = _tt(3, 6, 3)
    w = inputs.random_mpo(4, 6, 2, 3)
    probe = _tt(5, 6, 4)

    def loss():
        return core.inner(core.apply_mpo(w, x), probe)

    y = core.apply_mpo(w, x)
    dy, _ = grad.inner_vjp(y, probe, 1.0)
    dx, dw = grad.apply_mpo_vjp(w, x, dy)
    _fd_check(loss, x, dx)
    _fd_check(loss, w, dw, seed=2)


def test_hadamard_vjp_fd():
    x = _tt(6, 6, 3)
    y = _tt(7, 6, 2)
    probe = _tt(8, 6, 3)

    def loss():
        return core.inner(core.hadamard(x, y), probe)

    z = core.hadamard(x, y)
    dz, _ = grad.inner_vjp(z, probe, 1.0)
    dx, dy = grad.hadamard_vjp(x, y, dz)
    _fd_check(loss, x, dx)
    _fd_check(loss, y, dy, seed=3)


def test_evaluate_vjp_fd():
    x = _tt(9, 8, 4)
    digs = inputs.random_digits(10, 200, [2] * 8)
    w = np.random.default_rng(11).standard_normal(200)

    def loss():
        return float(np.dot(w, core.evaluate(x, digs)))

    g = grad.evaluate_vjp(x, digs, w)
    _fd_check(loss, x, g)


def test_fit_loss_grad_fd():
    bits = 4
    L = 2 * bits
    x = _tt(12, L, 3)
    digs = inputs.random_digits(13, 300, [2] * L)
    f = inputs.fit_targets(digs, bits)
    g = grad.fit_loss_grad(x, digs, f)
    _fd_check(lambda: grad.fit_loss(x, digs, f), x, g)


def test_residual_loss_grad_fd():
    from oracle import structured

    bits = 3
    w = structured.laplacian_mpo(2, bits)
    L = 2 * bits
    x = _tt(14, L, 3)
    b = _tt(15, L, 2)

    def loss():
        y = core.apply_mpo(w, x)
        f = core.full(y) - core.full(b)
        return float(np.sum(f * f))

    g = grad.residual_loss_grad(w, x, b)
    _fd_check(loss, x, g)


def test_inner_vjp_brute_force():
    """dX_k(i) from the adjoint equals the derivative of the full contraction (L = 4)."""
    x = _tt(16, 4, 2)
    y = _tt(17, 4, 3)
    dx, _ = grad.inner_vjp(x, y, 1.0)
    fy = core.full(y)
    # <x, y> is linear in X_2: contract everything else densely
    k = 2
    g = np.zeros_like(x[k])
    for idx in np.ndindex(*x[k].shape):
        e = [c.copy() for c in x]
        e[k] = np.zeros_like(x[k])
        e[k][idx] = 1.0
        g[idx] = np.sum(core.full(e) * fy)
    assert np.allclose(g, dx[k], rtol=1e-12, atol=1e-14)


# ---- the adjoint of rounding (Section 3.2's sweeps, reversed)


def _gap_train(seed, L):
    """A train with a clear gap in every unfolding spectrum: a rank-3 part plus 1e-5 times a
    rank-2 part (bond ranks 5, none above the ranks of the unfoldings)."""
    big = inputs.random_tt(seed, L, 2, [1, 2] + [3] * (L - 3) + [2, 1])
    small = inputs.random_tt(seed + 1, L, 2, [1] + [2] * (L - 1) + [1])
    return core.add(big, core.scale(small, 1e-5))


def test_round_vjp_without_truncation_is_the_inner_gradient():
    """No truncation: round(x) = x as a tensor, so the gradient of <round(x), y> is that of
    <x, y> (a closed form independent of the rounding's gauge)."""
    for L, ranks in [(4, [1, 2, 3, 2, 1]), (8, [1, 2, 4, 8, 9, 8, 4, 2, 1]), (6, [1, 2, 4, 3, 4, 2, 1])]:
        x = inputs.random_tt(11 + L, L, 2, ranks)
        y = inputs.random_tt(12 + L, L, 2, 3)
        dout, _ = grad.inner_vjp(core.round_tt(x, 1e-14), y)
        dx = grad.round_vjp(x, 1e-14, dout)
        ref, _ = grad.inner_vjp(x, y)
        scale = max(np.abs(r).max() for r in ref)
        for a, b in zip(dx, ref):
            assert np.abs(a - b).max() <= 1e-12 * scale


@pytest.mark.parametrize("eps", [1e-3, 1e-8])
def test_round_vjp_fd(eps):
    """<round(x), y> with truncation (eps = 1e-3 drops the 1e-5 part: ranks 5 -> 3) and
    without (eps = 1e-8), against central differences."""
    L = 7
    x = _gap_train(21, L)
    y = inputs.random_tt(23, L, 2, 3)
    out = core.round_tt(x, eps)
    assert max(core.ranks(out)) == (3 if eps == 1e-3 else 5)
    dout, _ = grad.inner_vjp(out, y)
    dx = grad.round_vjp(x, eps, dout)
    _fd_check(lambda: core.inner(core.round_tt(x, eps), y), x, dx)


def test_round_vjp_fd_norm_loss():
    """A second loss, ||round(x) - b||^2 for a fixed train b, through the same adjoint."""
    L = 6
    x = _gap_train(31, L)
    b = inputs.random_tt(33, L, 2, 2)

    def loss():
        z = core.round_tt(x, 1e-3)
        return core.inner(z, z) - 2.0 * core.inner(z, b)

    z = core.round_tt(x, 1e-3)
    d1, d2 = grad.inner_vjp(z, z)
    d3, _ = grad.inner_vjp(z, b, -2.0)
    dout = [p + q + r for p, q, r in zip(d1, d2, d3)]
    _fd_check(loss, x, grad.round_vjp(x, 1e-3, dout))
