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
        left.append(np.einsum("ab,aic,bid->cd", left[-1], x[k], y[k], optimize=True))
    right = [None] * (L + 1)
    right[L] = np.ones((1, 1))
    for k in range(L - 1, -1, -1):
        right[k] = np.einsum("aic,cd,bid->ab", x[k], right[k + 1], y[k], optimize=True)
    dx, dy = [], []
    for k in range(L):
        el, er = left[k], right[k + 1]
        dx.append(dout * np.einsum("ab,bid,cd->aic", el, y[k], er, optimize=True))
        dy.append(dout * np.einsum("ab,aic,cd->bid", el, x[k], er, optimize=True))
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


# ----------------------------------------------------------------------------
# adjoint of TT rounding (Section 3.2: the right-to-left orthogonalisation, then the
# left-to-right truncated decompositions)
# ----------------------------------------------------------------------------


def _copyltu(m):
    """Lower triangle copied to the upper one: tril(M) + tril(M, -1)^T."""
    lo = np.tril(m)
    return lo + np.tril(m, -1).T


def _qr_vjp(a, q, r, dq, dr):
    """Adjoint of the thin QR a = q r of an m x n matrix (Householder, numpy's convention).

    m >= n:  M = r dr^T - dq^T q,  da = (dq + q copyltu(M)) r^{-T}.
    m <  n:  a = q [r1 r2] = [x y] with r1 square: dy = q dr2, and x = q r1 takes the
             square rule with dq + y dr2^T in place of dq.
    Needs the square part of r to be invertible (the factorised matrix of full rank).
    """
    m, n = a.shape
    if m >= n:
        mm = r @ dr.T - dq.T @ q
        rhs = dq + q @ _copyltu(mm)
        return np.linalg.solve(r, rhs.T).T  # rhs r^{-T}
    r1, r2 = r[:, :m], r[:, m:]
    dr1, dr2 = dr[:, :m], dr[:, m:]
    y = a[:, m:]
    dy = q @ dr2
    dx = _qr_vjp(a[:, :m], q, r1, dq + y @ dr2.T, dr1)
    return np.hstack([dx, dy])


def _left_vectors_vjp(a, u, s, rn, db, guard):
    """Adjoint of b = u[:, :rn], the leading rn left singular vectors of a = u diag(s) v^T
    (thin SVD, m x n, s descending), given db (m x rn).

    With dU = [db, 0] and F_ij = 1 / (s_j^2 - s_i^2) (0 on the diagonal), the derivative of
    the SVD (the standard perturbation formula of the singular vectors) gives
        da = u [(F o (u^T dU - dU^T u)) S] v^T + (I - u u^T) dU S^{-1} v^T,
    and since S v^T = u^T a, with the columns of zero singular values left out,
        da = u (F o M) u^T a + (I - u u^T) db S_r^{-2} b^T a.
    Near-degenerate pairs (|s_i^2 - s_j^2| <= guard s_1^2) get F_ij = 0: for a loss that does
    not depend on the gauge of the kept basis their contributions cancel.
    """
    m, k = u.shape
    du = np.zeros((m, k))
    du[:, :rn] = db
    mm = u.T @ du - du.T @ u
    s2 = s * s
    diff = s2[None, :] - s2[:, None]  # s_j^2 - s_i^2
    tiny = guard * (s2[0] if k else 0.0)
    with np.errstate(divide="ignore"):
        f = np.where(np.abs(diff) > tiny, 1.0 / np.where(diff == 0.0, 1.0, diff), 0.0)
    np.fill_diagonal(f, 0.0)
    live = (s > 0.0).astype(np.float64)
    g = (f * mm) * live[None, :]
    da = u @ (g @ (u.T @ a))
    if m > k or rn > 0:
        b = u[:, :rn]
        x = db - u @ (u.T @ db)
        sr = s[:rn]
        inv2 = np.where(sr > 0.0, 1.0 / np.where(sr > 0.0, sr * sr, 1.0), 0.0)
        da += (x * inv2[None, :]) @ (b.T @ a)
    return da


def round_vjp(x, eps, dout, max_rank=None, guard=1e-13):
    """Gradient of a loss of round_tt(x, eps) w.r.t. the cores of x, given its gradient dout
    w.r.t. the output cores that core.round_tt(x, eps, max_rank) returns (the reverse of the
    two sweeps of round_tt; its forward steps are repeated exactly, so dout refers to the
    same gauge).

    Forward, as in round_tt: right-to-left, D_k^T = Q_k R_k, C_k = Q_k^T, D_{k-1} = x_{k-1} R_k^T
    (contracting the right bond); then left-to-right, with A_k the current core k as a matrix,
    B_k = its leading r'_k left singular vectors (the oracle's QR + SVD of R gives the same
    subspace), C_k = B_k and A_{k+1} = (B_k^T A_k) C_{k+1}.  The reverse runs the
    left-to-right sweep backwards (the adjoint of F = B^T A, of B = U_r(A) and of the product
    with the next core), then the right-to-left sweep forwards (the QR adjoints).

    Defined where the truncation ranks do not change under small perturbations (a gap at every
    cut) and every right-to-left factor is of full rank (bond ranks of x not above the ranks
    of its unfoldings).  The loss should not depend on the gauge of the output cores (e.g. a
    function of the represented tensor); near-degenerate kept singular values are guarded.
    """
    from .core import truncation_rank

    L = len(x)
    c = [np.array(g, dtype=np.float64, copy=True) for g in x]
    rl = [None] * L
    for k in range(L - 1, 0, -1):
        r0, d, r1 = c[k].shape
        dt = c[k].reshape(r0, d * r1).T.copy()
        q, rr = np.linalg.qr(dt)
        rl[k] = (dt, q, rr, c[k - 1].copy())
        p = q.shape[1]
        c[k] = np.ascontiguousarray(q.T).reshape(p, d, r1)
        c[k - 1] = np.einsum("adb,pb->adp", c[k - 1], rr)
    crl = [g.copy() for g in c]
    nrm = float(np.linalg.norm(c[0]))
    lr = [None] * L
    if L > 1:
        delta = eps * nrm / np.sqrt(L - 1)
        for k in range(L - 1):
            r0, d, r1 = c[k].shape
            # the steps of round_tt exactly (QR, SVD of R), so that the output cores, and the
            # gauge that dout refers to, are the same: u = q u_R are the left singular
            # vectors of a, and f = (S V^T)[:r'] = b^T a
            a = c[k].reshape(r0 * d, r1)
            q, rr = np.linalg.qr(a)
            ur, s, vt = np.linalg.svd(rr, full_matrices=False)
            rn = truncation_rank(s, delta, max_rank)
            u = q @ ur
            b = u[:, :rn]
            f = s[:rn, None] * vt[:rn]
            lr[k] = (a, u, s, rn, b, f)
            c[k] = (q @ ur[:, :rn]).reshape(r0, d, rn)
            c[k + 1] = np.einsum("ab,bdc->adc", f, c[k + 1])
    # ---- reverse of the left-to-right sweep
    dcrl = [None] * L
    g = np.array(dout[L - 1], dtype=np.float64)
    for k in range(L - 2, -1, -1):
        a, u, s, rn, b, f = lr[k]
        nxt = crl[k + 1]
        n1, d1, r2 = nxt.shape
        gm = g.reshape(rn, d1 * r2)
        df = gm @ nxt.reshape(n1, d1 * r2).T
        dcrl[k + 1] = (f.T @ gm).reshape(n1, d1, r2)
        db = np.asarray(dout[k], dtype=np.float64).reshape(b.shape) + a @ df.T
        da = b @ df + _left_vectors_vjp(a, u, s, rn, db, guard)
        g = da.reshape(a.shape[0] // crl[k].shape[1], crl[k].shape[1], a.shape[1])
    dcrl[0] = g.reshape(crl[0].shape)
    # ---- reverse of the right-to-left sweep
    dx = [None] * L
    dd = dcrl[0]  # cotangent of D_0 (= C_0 after the sweep)
    for k in range(1, L):
        dt, q, rr, xprev = rl[k]
        # D_{k-1} = xprev . rr^T over the right bond
        dx[k - 1] = np.einsum("adp,pb->adb", dd, rr)
        drr = np.einsum("adp,adb->pb", dd, xprev)
        p = q.shape[1]
        dq = dcrl[k].reshape(p, -1).T
        ddt = _qr_vjp(dt, q, rr, dq, drr)
        r0 = dt.shape[1]
        dd = ddt.T.reshape(r0, x[k].shape[1], -1)
    dx[L - 1] = dd.reshape(x[L - 1].shape)
    return dx
