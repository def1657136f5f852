"""FP64 oracle: the approximate einsums of Sections 3.2 and 3.3 for the MPO-TT product y = W x.

TEST INFRASTRUCTURE ONLY (see oracle/core.py).

decomposition_apply (Section 3.2, "decomposition algorithms", the zip-up of its figure)
    Both operands move their normalisation centre to the left end.  The exact product cores
    Y_1 .. Y_N of the first N sites (Y_k = the core-by-core product of apply_mpo) are contracted
    into a super-core C(i_1, .., i_N); a truncated SVD splits off C(i_1) (orthonormal columns)
    and leaves S V^T as the new super-core C(i_2, .., i_N), which is extended by the next exact
    product core, split again, and so on until no core is left.  The SVD split keeps the centre
    on the remaining super-core, so no extra QR is needed.  The threshold is
    delta = eps ||C(i_1..i_N)|| / sqrt(L - 1) with the norm of the first super-core (the paper
    states that with the centres at the left end the norm of the result depends only on it;
    that holds exactly when the super-core spans the whole train, N = L).
    Parity unpinned for N < L beyond exactness without truncation and the rank cap: the result
    has no closed form there, and the move of the operands' centres to the left end is pinned
    by no value (it changes nothing in the exact and N = L cases).

variational_apply (Section 3.3, Eq. (variational))
    C is kept in mixed canonical form with its centre on a super-core of N = ncores adjacent
    sites.  The update of the centre is the derivative of <C | y> with respect to it:
    C(i_q, .., i_{q+N-1}) = E^L_{q-1} Y_q .. Y_{q+N-1} E^R_{q+N}, where E^L and E^R are the
    environments of <C | y> over the sites left and right of the super-core (C's cores there
    orthonormal).  N = 2: the updated super-core is split by a truncated SVD (eps relative to its
    norm, max_rank), which moves the centre one site in the sweep direction and adapts the
    ranks.  N = 1: the core is replaced and the centre moved by a QR.  A sweep runs left to
    right and back.
"""
from __future__ import annotations

import math

import numpy as np

from . import core


def _mpo_orthogonalize_rl(w):
    """MPO cores (a, i, j, a') with the normalisation centre moved to the left end (the cores
    viewed as TT cores of mode i*j)."""
    t = [g.reshape(g.shape[0], g.shape[1] * g.shape[2], g.shape[3]) for g in w]
    t = core.orthogonalize_rl(t)
    return [c.reshape(c.shape[0], g.shape[1], g.shape[2], c.shape[2]) for c, g in zip(t, w)]


def decomposition_apply(w, x, eps, max_rank=None, ncores=2):
    """Zip-up approximation of W x with a super-core of ncores (1 <= ncores <= L) sites."""
    L = len(x)
    if L != len(w):
        raise ValueError("length mismatch")
    n_sc = max(1, min(int(ncores), L))
    y = core.apply_mpo(_mpo_orthogonalize_rl(w), core.orthogonalize_rl(x))
    # first super-core: (1, d_1, .., d_N, R_N)
    sc = y[0]
    for k in range(1, n_sc):
        sc = np.tensordot(sc, y[k], axes=([sc.ndim - 1], [0]))
    if L == 1:
        return [sc]
    delta = eps * float(np.linalg.norm(sc)) / math.sqrt(L - 1)
    out = []
    nxt = n_sc
    for k in range(L - 1):
        left, d = sc.shape[0], sc.shape[1]
        m = sc.reshape(left * d, -1)
        u, s, vt = np.linalg.svd(m, full_matrices=False)
        rn = core.truncation_rank(s, delta, max_rank)
        out.append(u[:, :rn].reshape(left, d, rn))
        sc = (s[:rn, None] * vt[:rn]).reshape((rn,) + sc.shape[2:])
        if nxt < L:  # extend the super-core by the next exact product core
            sc = np.tensordot(sc, y[nxt], axes=([sc.ndim - 1], [0]))
            nxt += 1
    out.append(sc.reshape(sc.shape[0], sc.shape[1], 1))
    return out


def _left_env(c, y, k):
    """E^L_k = sum over sites < k of C^T .. Y (shape r^C_k x r^Y_k); E^L_0 = 1."""
    e = np.ones((1, 1))
    for p in range(k):
        e = np.einsum("ab,aic,bid->cd", e, c[p], y[p], optimize=True)
    return e


def _right_env(c, y, k):
    """E^R_k = sum over sites >= k of C .. Y^T (shape r^C_k x r^Y_k); E^R_L = 1."""
    e = np.ones((1, 1))
    for p in range(len(c) - 1, k - 1, -1):
        e = np.einsum("aic,cd,bid->ab", c[p], e, y[p], optimize=True)
    return e


def _local_update(c, y, q, n):
    """d<C|y>/dC(i_q .. i_{q+n-1}) = E^L_q Y_q .. Y_{q+n-1} (E^R_{q+n})^T."""
    t = _left_env(c, y, q)  # (rC_q, rY_q)
    for p in range(q, q + n):
        t = np.tensordot(t, y[p], axes=([t.ndim - 1], [0]))
    er = _right_env(c, y, q + n)  # (rC_{q+n}, rY_{q+n})
    return np.tensordot(t, er, axes=([t.ndim - 1], [1]))  # (rC_q, d.., rC_{q+n})


def variational_apply(w, x, c0, nsweeps=2, ncores=2, eps=0.0, max_rank=None, trace=None):
    """Fit C to y = W x by sweeps of local updates (Eq. (variational)), starting from c0.

    trace: optional list that receives ||C - y|| after every local update (from the exact
    block sum, so it needs no full tensor)."""
    y = core.apply_mpo(w, x)
    L = len(y)
    n = 1 if L == 1 else max(1, min(int(ncores), 2))
    c = core.orthogonalize_rl(c0)  # centre at the left end
    if L == 1:
        c = [_local_update(c, y, 0, 1)]
        if trace is not None:
            trace.append(_dist(c, y))
        return c

    def split(sc, q, left_to_right):
        r0, r1 = sc.shape[0], sc.shape[-1]
        d0, d1 = sc.shape[1], sc.shape[2]
        m = sc.reshape(r0 * d0, d1 * r1)
        u, s, vt = np.linalg.svd(m, full_matrices=False)
        nrm = float(np.linalg.norm(s))
        rn = core.truncation_rank(s, eps * nrm, max_rank)
        if left_to_right:
            c[q] = u[:, :rn].reshape(r0, d0, rn)
            c[q + 1] = (s[:rn, None] * vt[:rn]).reshape(rn, d1, r1)
        else:
            c[q] = (u[:, :rn] * s[None, :rn]).reshape(r0, d0, rn)
            c[q + 1] = vt[:rn].reshape(rn, d1, r1)

    for _ in range(nsweeps):
        if n == 2:
            for q in range(0, L - 1):  # left to right; the centre ends on site L
                split(_local_update(c, y, q, 2), q, True)
                if trace is not None:
                    trace.append(_dist(c, y))
            for q in range(L - 2, -1, -1):  # right to left; the centre ends on site 1
                split(_local_update(c, y, q, 2), q, False)
                if trace is not None:
                    trace.append(_dist(c, y))
        else:
            for q in range(0, L):
                c[q] = _local_update(c, y, q, 1)
                if trace is not None:
                    trace.append(_dist(c, y))
                if q < L - 1:  # move the centre right: C_q = Q R, C_{q+1} <- R C_{q+1}
                    r0, d, r1 = c[q].shape
                    qm, rm = np.linalg.qr(c[q].reshape(r0 * d, r1))
                    c[q] = qm.reshape(r0, d, qm.shape[1])
                    c[q + 1] = np.einsum("ab,bdc->adc", rm, c[q + 1])
            for q in range(L - 1, -1, -1):
                c[q] = _local_update(c, y, q, 1)
                if trace is not None:
                    trace.append(_dist(c, y))
                if q > 0:  # move the centre left: C_q = L Q (QR of C_q^T), C_{q-1} <- C_{q-1} L
                    r0, d, r1 = c[q].shape
                    qm, rm = np.linalg.qr(c[q].reshape(r0, d * r1).T)
                    c[q] = qm.T.reshape(qm.shape[1], d, r1)
                    c[q - 1] = np.einsum("adb,pb->adp", c[q - 1], rm)
    return c


def _dist(c, y):
    return core.norm(core.add(c, core.scale(y, -1.0)))
