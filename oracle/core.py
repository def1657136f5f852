"""FP64 oracle: tensor-train arithmetic written out from its definitions.

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this module; only the
tests, the smoke check and the CPU-baseline leg of the benchmark may call it.
It shares no code with the CUDA path.

Plain numpy in float64 (complex128 where the cores are complex: the rounding of the Fourier
TT of Section 4.3).  A library primitive (matmul/einsum, Householder QR via
LAPACK geqrf/orgqr, SVD via LAPACK) serves as a single step; no blocking, fusion
or reordering is added beyond the definitions below.

Conventions
  * TT core G_k has shape (r_{k-1}, d_k, r_k), r_0 = r_L = 1 (Section 2, Eq. (vector_dec)).
  * MPO core W_k has shape (a_{k-1}, d_k(out i), d_k(in j), a_k).
  * Site 1 is the most significant digit, i = sum_q c_q i_q, c_q = prod_{r>q} b_r
    (Section 2, Eq. (quantization)); indices are 0-based.
  * Bond flattening after an einsum is xi = (mu, nu) with the first operand major,
    xi = mu * R_second + nu (Section 3.1, text after Eq. (einsum)).
"""
from __future__ import annotations

import math

import numpy as np

# ----------------------------------------------------------------------------
# shapes and full tensors
# ----------------------------------------------------------------------------


def ranks(x):
    """Bond ranks [r_0, ..., r_L] of a TT or MPO."""
    return [x[0].shape[0]] + [c.shape[-1] for c in x]


def dims(x):
    return [c.shape[1] for c in x]


def full(x):
    """Full tensor of a TT by contracting all bonds (Section 2, Eq. (vector_dec)).

    Returns an array of shape (d_1, ..., d_L); flattening it in C order gives the
    vector indexed by i = sum_q c_q i_q.
    """
    t = x[0]  # (1, d1, r1)
    for c in x[1:]:
        t = np.tensordot(t, c, axes=([t.ndim - 1], [0]))
    return t.reshape(t.shape[1:-1])


def full_mpo(w):
    """Dense matrix M[i, j] of an MPO; i and j are the flat output / input indices."""
    t = w[0]  # (1, d, d, a)
    for c in w[1:]:
        t = np.tensordot(t, c, axes=([t.ndim - 1], [0]))
    t = t.reshape(t.shape[1:-1])  # (i1, j1, i2, j2, ...)
    L = len(w)
    perm = [2 * k for k in range(L)] + [2 * k + 1 for k in range(L)]
    t = t.transpose(perm)
    n_out = int(np.prod([c.shape[1] for c in w]))
    n_in = int(np.prod([c.shape[2] for c in w]))
    return t.reshape(n_out, n_in)


# ----------------------------------------------------------------------------
# exact operations (Section 3.1)
# ----------------------------------------------------------------------------


def apply_mpo(w, x):
    """Exact 'ij,j->i' of an MPO and a TT, core by core (Eq. (quant_sum), Eq. (einsum)).

    Y_k[(a, r), i, (a', r')] = sum_j W_k[a, i, j, a'] G_k[r, j, r'],
    flattened with the operator bond major: xi = a * R_x + r.
    """
    if len(w) != len(x):
        raise ValueError("length mismatch")
    out = []
    for wk, gk in zip(w, x):
        a0, di, dj, a1 = wk.shape
        r0, dg, r1 = gk.shape
        if dj != dg:
            raise ValueError("mode mismatch")
        y = np.einsum("aijb,rjs->aribs", wk, gk)
        out.append(y.reshape(a0 * r0, di, a1 * r1))
    return out


def hadamard(x, y):
    """Exact 'i,i->i' of two TTs (Eq. (einsum) with the index kept, not summed).

    Z_k[(r, s), i, (r', s')] = X_k[r, i, r'] Y_k[s, i, s'], first operand major.
    """
    if len(x) != len(y):
        raise ValueError("length mismatch")
    out = []
    for xk, yk in zip(x, y):
        r0, d, r1 = xk.shape
        s0, e, s1 = yk.shape
        if d != e:
            raise ValueError("mode mismatch")
        z = np.einsum("ria,sib->rsiab", xk, yk)
        out.append(z.reshape(r0 * s0, d, r1 * s1))
    return out


def add(x, y):
    """Exact sum with block cores (Section 3.1, the block equation for A + B).

    First core [A B], middle cores diag(A, B), last core [A; B].
    """
    L = len(x)
    if L != len(y):
        raise ValueError("length mismatch")
    if L == 1:
        return [x[0] + y[0]]
    out = []
    for k in range(L):
        a, b = x[k], y[k]
        ra0, d, ra1 = a.shape
        rb0, _, rb1 = b.shape
        if k == 0:
            c = np.zeros((1, d, ra1 + rb1))
            c[:, :, :ra1] = a
            c[:, :, ra1:] = b
        elif k == L - 1:
            c = np.zeros((ra0 + rb0, d, 1))
            c[:ra0] = a
            c[ra0:] = b
        else:
            c = np.zeros((ra0 + rb0, d, ra1 + rb1))
            c[:ra0, :, :ra1] = a
            c[ra0:, :, ra1:] = b
        out.append(c)
    return out


def scale(x, alpha):
    out = [c.copy() for c in x]
    out[0] = out[0] * alpha
    return out


def inner(x, y):
    """<x, y> with every index contracted ('i,i->'), by the left environment sweep.

    E_0 = 1, E_k = sum_i X_k(i)^T E_{k-1} Y_k(i); <x, y> = E_L.  The three-factor sum is
    contracted pairwise (optimize=True: O(r^3) per site instead of the O(r^4) of a joint loop
    over all five indices).
    """
    e = np.ones((1, 1))
    for xk, yk in zip(x, y):
        e = np.einsum("ab,aic,bid->cd", e, xk, yk, optimize=True)
    return float(e[0, 0])


def evaluate(x, digits):
    """Entries x(i_1, ..., i_L) at n digit tuples (exact sampling): v_s = prod_k G_k[:, i_k^s, :]."""
    digits = np.asarray(digits)
    n = digits.shape[0]
    v = np.ones((n, 1))
    for k, gk in enumerate(x):
        sl = gk[:, digits[:, k].astype(np.int64), :]  # (r0, n, r1)
        v = np.einsum("sa,asb->sb", v, sl)
    return v[:, 0]


# ----------------------------------------------------------------------------
# canonical form and rounding (Section 3.2; truncation threshold of TT rounding)
# ----------------------------------------------------------------------------


def orthogonalize_rl(x):
    """Move the normalisation centre to the left end (Section 3.2, first step).

    For k = L..2: LQ of C_k viewed as r_{k-1} x (d_k r_k) (as the QR of its
    transpose), C_k <- Q (orthonormal rows), C_{k-1} <- C_{k-1} L.
    Afterwards ||x|| = ||C_1||_F.
    """
    # float64, or complex128 for complex cores (the Fourier TT of Section 4.3); with complex
    # cores q^T still has orthonormal rows, so the same steps hold
    c = [np.array(g, dtype=np.result_type(g, np.float64), copy=True) for g in x]
    for k in range(len(c) - 1, 0, -1):
        r0, d, r1 = c[k].shape
        m = c[k].reshape(r0, d * r1)
        q, rr = np.linalg.qr(m.T)  # m^T = q rr, q: (d r1) x p, rr: p x r0
        p = q.shape[1]
        c[k] = np.ascontiguousarray(q.T).reshape(p, d, r1)
        c[k - 1] = np.einsum("adb,pb->adp", c[k - 1], rr)  # C_{k-1} rr^T
    return c


def norm(x):
    """Frobenius norm via the orthogonalisation sweep (no <x,x> cancellation)."""
    c = orthogonalize_rl(x)
    return float(np.linalg.norm(c[0]))


def truncation_rank(sigma, delta, max_rank=None):
    """Smallest r' >= 1 with (sum_{j > r'} sigma_j^2)^(1/2) <= delta, capped at max_rank.

    sigma is sorted descending.  The tail bound is inclusive.
    """
    n = len(sigma)
    tail2 = 0.0
    r = n
    # walk from the end while the accumulated tail stays within delta
    for j in range(n - 1, 0, -1):
        t = tail2 + sigma[j] * sigma[j]
        if math.sqrt(t) <= delta:
            tail2 = t
            r = j
        else:
            break
    r = max(r, 1)
    if max_rank is not None and max_rank > 0:
        r = min(r, int(max_rank))
    return r


def round_tt(x, eps, max_rank=None, return_info=False):
    """TT rounding: right-to-left orthogonalisation, then left-to-right truncated SVDs.

    Step order follows Section 3.2 (normalisation centre to the left end, then a
    decomposition at each bond while sliding right, re-normalising onto the next
    core).  The per-bond threshold is delta = eps * ||x|| / sqrt(L - 1), with
    ||x|| read off the orthogonalised first core; this guarantees
    ||x - round(x)|| <= eps ||x||.  At bond k:
        QR of C_k as (r_{k-1} d) x r_k  ->  Q, R
        SVD R = U S V^T (descending S)
        r' = truncation_rank(S, delta, max_rank)
        C_k <- Q U[:, :r'],   C_{k+1} <- (S V^T)[:r'] C_{k+1}.
    """
    L = len(x)
    c = orthogonalize_rl(x)
    nrm = float(np.linalg.norm(c[0]))
    info = {"norm": nrm, "sigmas": [], "ranks": None}
    if L == 1:
        info["ranks"] = ranks(c)
        return (c, info) if return_info else c
    delta = eps * nrm / math.sqrt(L - 1)
    for k in range(L - 1):
        r0, d, r1 = c[k].shape
        a = c[k].reshape(r0 * d, r1)
        q, rr = np.linalg.qr(a)
        u, s, vt = np.linalg.svd(rr, full_matrices=False)
        info["sigmas"].append(s.copy())
        rn = truncation_rank(s, delta, max_rank)
        c[k] = (q @ u[:, :rn]).reshape(r0, d, rn)
        sv = s[:rn, None] * vt[:rn]
        c[k + 1] = np.einsum("ab,bdc->adc", sv, c[k + 1])
    info["ranks"] = ranks(c)
    return (c, info) if return_info else c


def rel_err(a, b):
    """e(a, b) = ||a - b|| / ||b|| through the exact block sum a + (-b) (Section 3.1)."""
    nb = norm(b)
    diff = add(a, scale(b, -1.0))
    nd = norm(diff)
    return nd / nb if nb > 0 else nd


def left_orthogonality_defect(core):
    """||Q^T Q - I||_F for a core viewed as (r_{k-1} d) x r_k."""
    r0, d, r1 = core.shape
    q = core.reshape(r0 * d, r1)
    return float(np.linalg.norm(q.T @ q - np.eye(r1)))


def right_orthogonality_defect(core):
    """||Q Q^T - I||_F for a core viewed as r_{k-1} x (d r_k)."""
    r0, d, r1 = core.shape
    q = core.reshape(r0, d * r1)
    return float(np.linalg.norm(q @ q.T - np.eye(r0)))
