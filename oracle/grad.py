"""FP64 oracle: hand-derived adjoints of apply / hadamard / inner / eval.

TEST INFRASTRUCTURE ONLY (see oracle/core.py).  Each function returns the
vector-Jacobian product of the corresponding exact operation in oracle/core.py,
i.e. the gradient of a scalar loss with respect to the input cores given the
gradient with respect to the output.  The same environment algebra as the
derivative of an overlap with respect to one core (Section 3.3, Eq. (variational))
is used for inner and eval.  The tests pin every function against central finite
differences of the forward definition.
"""
from __future__ import annotations

import numpy as np


def apply_mpo_vjp(w, x, dy):
    """Adjoint of Y_k[(a,r), i, (a',r')] = sum_j W_k[a,i,j,a'] G_k[r,j,r'].

    dG_k[r, j, r'] = sum_{a, a', i} W_k[a, i, j, a'] dY_k[(a, r), i, (a', r')]
    dW_k[a, i, j, a'] = sum_{r, r'} G_k[r, j, r'] dY_k[(a, r), i, (a', r')]
    """
    dx, dw = [], []
    for wk, gk, dyk in zip(w, x, dy):
        a0, di, dj, a1 = wk.shape
        r0, _, r1 = gk.shape
        d5 = dyk.reshape(a0, r0, di, a1, r1)
        dx.append(np.einsum("aijb,aribs->rjs", wk, d5))
        dw.append(np.einsum("rjs,aribs->aijb", gk, d5))
    return dx, dw


def hadamard_vjp(x, y, dz):
    """Adjoint of Z_k[(r,s), i, (r',s')] = X_k[r,i,r'] Y_k[s,i,s']."""
    dx, dy = [], []
    for xk, yk, dzk in zip(x, y, dz):
        r0, d, r1 = xk.shape
        s0, _, s1 = yk.shape
        d5 = dzk.reshape(r0, s0, d, r1, s1)
        dx.append(np.einsum("rsiab,sib->ria", d5, yk))
        dy.append(np.einsum("rsiab,ria->sib", d5, xk))
    return dx, dy


def inner_vjp(x, y, dout=1.0):
    """Gradient of <x, y> w.r.t. the cores of x and y.

    With left environments E^L_k (E^L_0 = 1) and right environments E^R_k
    (E^R_L = 1, E^R_{k-1} = sum_i X_k(i) E^R_k Y_k(i)^T):
        dX_k(i) = dout * E^L_{k-1} Y_k(i) (E^R_k)^T
        dY_k(i) = dout * (E^L_{k-1})^T X_k(i) E^R_k
    """
    L = len(x)
    left = [np.ones((1, 1))]
    for k in range(L):
        left.append(np.einsum("ab,aic,bid->cd", left[-1], x[k], y[k]))
    right = [None] * (L + 1)
    right[L] = np.ones((1, 1))
    for k in range(L - 1, -1, -1):
        right[k] = np.einsum("aic,cd,bid->ab", x[k], right[k + 1], y[k])
    dx, dy = [], []
    for k in range(L):
        el, er = left[k], right[k + 1]
        dx.append(dout * np.einsum("ab,bid,cd->aic", el, y[k], er))
        dy.append(dout * np.einsum("ab,aic,cd->bid", el, x[k], er))
    return dx, dy


def evaluate_vjp(x, digits, dvals):
    """Gradient of sum_s dvals_s * x(i^s) w.r.t. the cores.

    dG_k[:, i, :] = sum_{s : i_k^s = i} dvals_s * prefix_s^T suffix_s, with
    prefix_s = G_1[:, i_1^s, :] ... G_{k-1}[:, i_{k-1}^s, :] (row vector) and
    suffix_s = G_{k+1}[:, i_{k+1}^s, :] ... G_L[:, i_L^s, :] (column vector).
    """
    digits = np.asarray(digits).astype(np.int64)
    n = digits.shape[0]
    L = len(x)
    pre = [np.ones((n, 1))]
    for k in range(L):
        pre.append(np.einsum("sa,asb->sb", pre[-1], x[k][:, digits[:, k], :]))
    suf = [None] * (L + 1)
    suf[L] = np.ones((n, 1))
    for k in range(L - 1, -1, -1):
        suf[k] = np.einsum("asb,sb->sa", x[k][:, digits[:, k], :], suf[k + 1])
    grads = []
    dv = np.asarray(dvals, dtype=np.float64)
    for k in range(L):
        r0, d, r1 = x[k].shape
        g = np.zeros((r0, d, r1))
        outer = np.einsum("s,sa,sb->sab", dv, pre[k], suf[k + 1])
        for i in range(d):
            m = digits[:, k] == i
            if m.any():
                g[:, i, :] = outer[m].sum(axis=0)
        grads.append(g)
    return grads


def fit_loss(x, digits, targets):
    """l = 1/(2N) sum_s (x(i^s) - f_s)^2, the sample-fit loss."""
    from .core import evaluate

    v = evaluate(x, digits)
    n = len(targets)
    return 0.5 * float(np.sum((v - targets) ** 2)) / n


def fit_loss_grad(x, digits, targets):
    from .core import evaluate

    v = evaluate(x, digits)
    n = len(targets)
    return evaluate_vjp(x, digits, (v - targets) / n)


def residual_loss_grad(w, x, b):
    """Gradient of ||W x - b||^2 w.r.t. the cores of x.

    ||y - b||^2 = <y, y> - 2 <y, b> + <b, b> with y = W x; the gradient w.r.t. the
    cores of y is 2 d<y,y>/2 ... composed through the apply adjoint.
    """
    from .core import apply_mpo

    y = apply_mpo(w, x)
    dyy, _ = inner_vjp(y, y, 1.0)  # d<y,y>/dY through the first slot
    _, dyy2 = inner_vjp(y, y, 1.0)  # ... and through the second slot
    dyb, _ = inner_vjp(y, b, -2.0)
    dy = [a + c + e for a, c, e in zip(dyy, dyy2, dyb)]
    dx, _ = apply_mpo_vjp(w, x, dy)
    return dx
