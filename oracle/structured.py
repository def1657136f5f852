"""FP64 oracle: structured tensors written out from Section 4.

TEST INFRASTRUCTURE ONLY (see oracle/core.py).  Closed-form TTs of exp, cos, sin
and polynomials on a uniform grid, the shift matrices Q^N_d / R^N_d as MPOs, and
the Dirichlet second-difference operators built from them.

Grid (Section 2): x(i) = (b - a)/(N - 1) * i + a, i = sum_q c_q i_q, so
x = sum_q c_q x_q + a with x_q = (b - a)/(N - 1) * i_q.
"""
from __future__ import annotations

import math

import numpy as np


def coefficients(bases):
    """c_q = prod_{r > q} b_r (Section 2, Eq. (quantization))."""
    n = len(bases)
    c = [1] * n
    for q in range(n - 2, -1, -1):
        c[q] = c[q + 1] * bases[q + 1]
    return c


def to_digits(idx, bases):
    """Flat indices -> digit tuples (most significant first)."""
    idx = np.asarray(idx, dtype=np.int64)
    c = coefficients(bases)
    out = np.empty(idx.shape + (len(bases),), dtype=np.int64)
    rem = idx.copy()
    for q, cq in enumerate(c):
        out[..., q] = rem // cq
        rem = rem - out[..., q] * cq
    return out


def to_idxs(digits, bases):
    c = coefficients(bases)
    digits = np.asarray(digits, dtype=np.int64)
    return (digits * np.asarray(c, dtype=np.int64)).sum(axis=-1)


def grid_points(bases, lower, upper):
    n_total = int(np.prod(bases))
    return lower + (upper - lower) / (n_total - 1) * np.arange(n_total)


def _digit_values(bases, lower, upper):
    """x_q values per site: (b - a)/(N - 1) * c_q * [0, 1, ..., b_q - 1]."""
    n_total = int(np.prod(bases))
    h = (upper - lower) / (n_total - 1)
    c = coefficients(bases)
    return [h * c[q] * np.arange(bases[q], dtype=np.float64) for q in range(len(bases))]


def exp_tt(bases, lower, upper, v, x0=0.0):
    """e^{v (x - x0)} as a rank-1 TT (Section 4.1, Eq. (exp_dec))."""
    xs = _digit_values(bases, lower, upper)
    cores = []
    for q, xq in enumerate(xs):
        vals = np.exp(v * xq)
        if q == 0:
            vals = vals * math.exp(v * (lower - x0))
        cores.append(vals.reshape(1, -1, 1))
    return cores


def cos_tt(bases, lower, upper, v, x0=0.0, phase=0.0):
    """cos(v (x - x0) + phase) as the real rank-2 rotation TT of Section 4.1.

    cos(Theta) = 1/2 (1, 1) prod_q Rot(xt_q) (1, 1)^T with Rot(t) = [[cos t, -sin t],
    [sin t, cos t]] and xt_q = v c_q x_q + (v (a - x0) + phase)/n, so sum_q xt_q = Theta.
    """
    xs = _digit_values(bases, lower, upper)
    n = len(bases)
    off = (v * (lower - x0) + phase) / n
    cores = []
    for q, xq in enumerate(xs):
        t = v * xq + off
        rot = np.empty((2, len(t), 2))
        rot[0, :, 0] = np.cos(t)
        rot[0, :, 1] = -np.sin(t)
        rot[1, :, 0] = np.sin(t)
        rot[1, :, 1] = np.cos(t)
        cores.append(rot)
    if n == 1:
        c = 0.5 * np.einsum("a,aib,b->i", np.ones(2), cores[0], np.ones(2))
        return [c.reshape(1, -1, 1)]
    first = 0.5 * np.einsum("a,aib->ib", np.ones(2), cores[0])
    last = np.einsum("aib,b->ai", cores[-1], np.ones(2))
    cores[0] = first.reshape(1, -1, 2)
    cores[-1] = last.reshape(2, -1, 1)
    return cores


def sin_tt(bases, lower, upper, v, x0=0.0):
    """sin(v (x - x0)) = cos(v (x - x0) - pi/2): the rotation TT shifted by pi/2 (Section 4.1)."""
    return cos_tt(bases, lower, upper, v, x0, phase=-0.5 * math.pi)


def poly_tt(bases, lower, upper, coeffs, x0=0.0):
    """sum_s v_s (x - x0)^s as a TT of rank p + 1 (Section 4.1, polynomials).

    xt_q = c_q x_q + (a - x0)/n.  First core: entry u = sum_{t >= u} v_t C(t, u) xt_1^{t-u}.
    Middle core: entry [s][u] = C(s, u) xt_q^{s-u} for u <= s (left bond s, right bond u).
    Last core: entry s = xt_n^s.  (The printed middle core has its bond indices
    transposed relative to the first and last cores; this orientation is the one
    that reproduces f, as the brute-force test checks.)
    """
    xs = _digit_values(bases, lower, upper)
    n = len(bases)
    p = len(coeffs) - 1
    off = (lower - x0) / n
    binom = [[math.comb(s, u) for u in range(p + 1)] for s in range(p + 1)]
    cores = []
    for q, xq in enumerate(xs):
        t = xq + off
        b = len(t)
        if q == 0:
            c = np.zeros((1, b, p + 1))
            for u in range(p + 1):
                acc = np.zeros(b)
                for tt in range(u, p + 1):
                    acc += coeffs[tt] * binom[tt][u] * t ** (tt - u)
                c[0, :, u] = acc
            if n == 1:
                # single site: contract with the last-core vector xt^s at xt = 0 -> keep u = 0
                return [c[:, :, :1]]
        elif q == n - 1:
            c = np.zeros((p + 1, b, 1))
            for s in range(p + 1):
                c[s, :, 0] = t ** s
        else:
            c = np.zeros((p + 1, b, p + 1))
            for s in range(p + 1):
                for u in range(s + 1):
                    c[s, :, u] = binom[s][u] * t ** (s - u)
        cores.append(c)
    return cores


# ----------------------------------------------------------------------------
# shift matrices and operators (Section 4.2, Eq. (shif_dec))
# ----------------------------------------------------------------------------


def q_shift(b, d):
    """Q^b_d(i, j) = 1 iff i - j = d (zero matrix when d >= b)."""
    m = np.zeros((b, b))
    for i in range(b):
        j = i - d
        if 0 <= j < b:
            m[i, j] = 1.0
    return m


def r_shift(b, d):
    """R^b_d = (Q^b_{b-d})^T, i.e. R(i, j) = 1 iff i - j = d - b."""
    return q_shift(b, b - d).T if b - d >= 0 else np.zeros((b, b))


def shift_digits(bases, d):
    """Greedy digits of the shift d = sum_q c_q d_q.

    The printed recursion subtracts a product of earlier terms; the digits of a
    mixed-radix number need their sum, which is what is used here.
    """
    c = coefficients(bases)
    out = []
    rem = d
    for cq in c:
        out.append(rem // cq)
        rem -= out[-1] * cq
    return out


def shift_mpo(bases, d):
    """Q^N_d as a rank-2 MPO from the iterated rank product of Eq. (shif_dec).

    Core q (state 0 = "Q", state 1 = "R"):
        [[Q^{b_q}_{d_q}, Q^{b_q}_{d_q+1}], [R^{b_q}_{d_q}, R^{b_q}_{d_q+1}]],
    the last core is the column [Q^{b_n}_{d_n}; R^{b_n}_{d_n}], and the row vector
    (1, 0) on the left selects Q^N_d.
    """
    n = len(bases)
    dq = shift_digits(bases, d)
    cores = []
    for q in range(n):
        b = bases[q]
        blocks = [[q_shift(b, dq[q]), q_shift(b, dq[q] + 1)],
                  [r_shift(b, dq[q]), r_shift(b, dq[q] + 1)]]
        if q == n - 1:
            c = np.zeros((2, b, b, 1))
            c[0, :, :, 0] = blocks[0][0]
            c[1, :, :, 0] = blocks[1][0]
        else:
            c = np.zeros((2, b, b, 2))
            for s in range(2):
                for t in range(2):
                    c[s, :, :, t] = blocks[s][t]
        cores.append(c)
    cores[0] = cores[0][:1]  # (1, 0) from the left
    return cores


def mpo_transpose(w):
    return [np.ascontiguousarray(c.transpose(0, 2, 1, 3)) for c in w]


def mpo_identity(bases):
    return [np.eye(b).reshape(1, b, b, 1) for b in bases]


def mpo_add(w1, w2):
    """Exact MPO sum with block cores (Section 3.1 applied to operator cores)."""
    L = len(w1)
    if L == 1:
        return [w1[0] + w2[0]]
    out = []
    for k in range(L):
        a, b = w1[k], w2[k]
        ra0, di, dj, ra1 = a.shape
        rb0, _, _, rb1 = b.shape
        if k == 0:
            c = np.zeros((1, di, dj, ra1 + rb1))
            c[..., :ra1] = a
            c[..., ra1:] = b
        elif k == L - 1:
            c = np.zeros((ra0 + rb0, di, dj, 1))
            c[:ra0] = a
            c[ra0:] = b
        else:
            c = np.zeros((ra0 + rb0, di, dj, ra1 + rb1))
            c[:ra0, :, :, :ra1] = a
            c[ra0:, :, :, ra1:] = b
        out.append(c)
    return out


def mpo_scale(w, alpha):
    out = [c.copy() for c in w]
    out[0] = out[0] * alpha
    return out


def second_difference_sum_mpo(bases):
    """Q_1 + Q_1^T - 2 I as the exact block sum of three MPOs (rank 5).

    Dirichlet boundary (zero outside the grid), no 1/h^2 scaling.
    """
    q1 = shift_mpo(bases, 1)
    return mpo_add(mpo_add(q1, mpo_transpose(q1)), mpo_scale(mpo_identity(bases), -2.0))


def embed_mpo(w_dim, layout, dim):
    """Place a one-dimension MPO on the sites of dimension `dim` of an interleaved layout.

    layout[k] = dimension owning site k.  Sites of other dimensions carry the
    identity and pass the bond through unchanged.
    """
    out = []
    it = iter(w_dim)
    cur_rank = 1
    for k, owner in enumerate(layout):
        if owner == dim:
            c = next(it)
            cur_rank = c.shape[-1]
            out.append(c)
        else:
            b = 2
            c = np.zeros((cur_rank, b, b, cur_rank))
            for s in range(cur_rank):
                c[s, :, :, s] = np.eye(b)
            out.append(c)
    # fix the first core's left rank when the first site is not owned by `dim`
    # (bond rank 1 there already) and check consistency of the chain
    for k in range(1, len(out)):
        if out[k].shape[0] != out[k - 1].shape[-1]:
            raise ValueError("inconsistent embedding")
    return out


def interleaved_layout(n_dims, bits):
    """Site k holds bit k // n_dims of dimension k % n_dims (x_1, y_1, x_2, y_2, ...)."""
    return [k % n_dims for k in range(n_dims * bits)]


def laplacian_mpo_sum(n_dims, bits):
    """Kronecker-sum Dirichlet Laplacian on an interleaved binary layout, as an exact
    sum of embedded one-dimension second differences (rank 5 * n_dims, not minimal)."""
    layout = interleaved_layout(n_dims, bits)
    total = None
    for t in range(n_dims):
        e = embed_mpo(second_difference_sum_mpo([2] * bits), layout, t)
        total = e if total is None else mpo_add(total, e)
    return total


def laplacian_mpo(n_dims, bits):
    """Minimal-rank Dirichlet Laplacian MPO on an interleaved binary layout.

    Built as a finite-state operator from the shift structure of Eq. (shif_dec)
    (with Q^2_0 = I, Q^2_1 = J, R^2_1 = J^T, R^2_0 = 0):
      state 0       : identity so far, every term still pending;
      state (t, +)  : the +1 shift of dimension t has produced a carry (J^T pending);
      state (t, -)  : the -1 shift of dimension t has produced a carry (J pending);
      state done    : some dimension's term has finished, identity from here on.
    On the last site of dimension t: 0 -> done with J + J^T - 2I, (t,+) -> done
    with J^T, (t,-) -> done with J.  States that are unreachable or cannot reach
    the end are dropped, giving ranks 3 (1D), 5 (2D), 7 (3D).
    """
    layout = interleaved_layout(n_dims, bits)
    L = len(layout)
    J = q_shift(2, 1)
    Jt = J.T
    I = np.eye(2)
    states = ["0"] + [(t, s) for t in range(n_dims) for s in "+-"] + ["done"]
    S = len(states)
    idx = {s: i for i, s in enumerate(states)}
    last_site = {t: max(k for k in range(L) if layout[k] == t) for t in range(n_dims)}
    big = []
    for k in range(L):
        owner = layout[k]
        c = np.zeros((S, 2, 2, S))
        is_last = k == last_site[owner]
        # identity pass-through for states not touched by this site's dimension
        for s in states:
            if s == "0" or s == "done":
                continue
            if s[0] != owner:
                c[idx[s], :, :, idx[s]] = I
        c[idx["done"], :, :, idx["done"]] = I
        if not is_last:
            c[idx["0"], :, :, idx["0"]] = I
            c[idx["0"], :, :, idx[(owner, "+")]] = J
            c[idx["0"], :, :, idx[(owner, "-")]] = Jt
            c[idx[(owner, "+")], :, :, idx[(owner, "+")]] = Jt
            c[idx[(owner, "-")], :, :, idx[(owner, "-")]] = J
        else:
            # terms of other dimensions may still be pending: keep state 0
            pending_other = any(last_site[t] > k for t in range(n_dims) if t != owner)
            if pending_other:
                c[idx["0"], :, :, idx["0"]] = I
            c[idx["0"], :, :, idx["done"]] = J + Jt - 2 * I
            c[idx[(owner, "+")], :, :, idx["done"]] = Jt
            c[idx[(owner, "-")], :, :, idx["done"]] = J
        big.append(c)
    # boundary vectors: start in state 0, end in state done
    big[0] = big[0][idx["0"]:idx["0"] + 1]
    big[-1] = big[-1][..., idx["done"]:idx["done"] + 1]
    # prune states: reachable from the left and able to reach the right
    alive_left = [np.ones(1, dtype=bool)]
    for k in range(L):
        c = big[k]
        nz = np.abs(c).sum(axis=(1, 2)) > 0  # (left, right)
        reach = (nz & alive_left[-1][:, None]).any(axis=0)
        alive_left.append(reach)
    alive_right = [None] * (L + 1)
    alive_right[L] = np.ones(1, dtype=bool)
    for k in range(L - 1, -1, -1):
        c = big[k]
        nz = np.abs(c).sum(axis=(1, 2)) > 0
        alive_right[k] = (nz & alive_right[k + 1][None, :]).any(axis=1)
    keep = [alive_left[k] & alive_right[k] for k in range(L + 1)]
    out = []
    for k in range(L):
        c = big[k][keep[k]][..., keep[k + 1]]
        out.append(np.ascontiguousarray(c))
    return out


def dense_laplacian(n_dims, bits):
    """Dense Kronecker-sum Dirichlet Laplacian in natural (x, y, ...) index order."""
    n = 2 ** bits
    d1 = -2.0 * np.eye(n) + np.eye(n, k=1) + np.eye(n, k=-1)
    total = np.zeros((n ** n_dims, n ** n_dims))
    for t in range(n_dims):
        term = np.ones((1, 1))
        for s in range(n_dims):
            term = np.kron(term, d1 if s == t else np.eye(n))
        total += term
    return total


def interleaved_permutation(n_dims, bits):
    """perm[flat interleaved index] = flat natural (x, y, ...) index."""
    L = n_dims * bits
    n_total = 2 ** L
    flat = np.arange(n_total)
    digs = to_digits(flat, [2] * L)  # site digits, interleaved order
    nat = np.zeros(n_total, dtype=np.int64)
    for t in range(n_dims):
        coord = np.zeros(n_total, dtype=np.int64)
        for q in range(bits):
            coord = coord * 2 + digs[:, q * n_dims + t]
        nat = nat * (2 ** bits) + coord
    return nat
