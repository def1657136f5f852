"""FP64 oracle: the Fourier (DFT) matrix as a tensor train (Section 4.3).

TEST INFRASTRUCTURE ONLY (see oracle/core.py).  Complex128 throughout.

The DFT matrix of size N = prod_q b_q is M(i, j) = v^(i j) with v = exp(-2 pi i / N) (the
printed "v e^{ij}" read as the power v^{ij}).  Row indices are factorised most significant digit
first, i = sum_q c_q i_q with c_q = prod_{r > q} b_r (Section 2, Eq. (quantization)); column
indices use the REVERSED list of bases, so that core q carries i_q together with the column digit
of the same base, j_{n-q+1} (0-based: site p carries i_p and the column digit whose weight is
prod_{u < p} b_u, the least significant column digit on the first site).

Since i j = sum_q c_q i_q j, M is the element-wise product over q of T_q(i_q, j) = v^(c_q i_q j),
and T_q = sum_s delta(s, i_q) prod_p v^(s c_q w_p j_p) is a sum of b_q rank-one trains: an MPO of
rank b_q whose bond index s runs unchanged through every site.  The Fourier TT multiplies the n
factors one after the other, rounding after each element-wise product with the rank capped at
max_rank (the apply-then-round reading of the paper's zip-up multiplication).

Exponents are reduced modulo N in exact integer arithmetic before exp() is taken, so every
entry of every factor is correct to the last bit of its phase.
"""
from __future__ import annotations

import cmath
import math

import numpy as np

from . import core


def _weights(bases):
    """(row weights c_p, column weights w_p of the digit on site p)."""
    n = len(bases)
    c = [int(np.prod(bases[p + 1:], dtype=np.int64)) for p in range(n)]
    w = [int(np.prod(bases[:p], dtype=np.int64)) for p in range(n)]
    return c, w


def factor_mpo(bases, q):
    """T_q(i_q, j) = v^(c_q i_q j) as a rank-b_q MPO, cores of shape (s, i_p, j_p, s')."""
    n = len(bases)
    N = int(np.prod(bases, dtype=np.int64))
    c, w = _weights(bases)
    bq = bases[q]
    cores = []
    for p in range(n):
        b = bases[p]
        g = np.zeros((bq, b, b, bq), dtype=np.complex128)
        for s in range(bq):
            for jp in range(b):
                phase = cmath.exp(-2j * math.pi * ((s * c[q] * w[p] * jp) % N) / N)
                if p == q:
                    g[s, s, jp, s] = phase  # delta(s, i_q)
                else:
                    g[s, :, jp, s] = phase  # independent of i_p
        cores.append(g)
    cores[0] = cores[0].sum(axis=0, keepdims=True)    # sum over s from the left
    cores[-1] = cores[-1].sum(axis=3, keepdims=True)  # ... and close it on the right
    return cores


def _as_tt(w):
    """MPO cores (a, i, j, a') as TT cores (a, i*b + j, a')."""
    return [g.reshape(g.shape[0], g.shape[1] * g.shape[2], g.shape[3]) for g in w]


def _as_mpo(x, bases):
    return [g.reshape(g.shape[0], b, b, g.shape[2]) for g, b in zip(x, bases)]


def fourier_mpo(bases, max_rank=None, eps=0.0):
    """The Fourier TT: T_1 (.) T_2 (.) ... (.) T_n, each element-wise product rounded at once
    (eps, and bond ranks capped at max_rank).  max_rank=None and eps=0 give the exact product."""
    x = _as_tt(factor_mpo(bases, 0))
    for q in range(1, len(bases)):
        x = core.hadamard(x, _as_tt(factor_mpo(bases, q)))
        if max_rank is not None or eps > 0.0:
            x = core.round_tt(x, eps, max_rank)
    return _as_mpo(x, bases)


def dense(w, bases):
    """The N x N matrix of a Fourier-layout MPO: rows from the i digits (site order), columns
    from the j digits (site p holds the digit of weight prod_{u < p} b_u)."""
    n = len(bases)
    t = w[0]
    for g in w[1:]:
        t = np.tensordot(t, g, axes=([t.ndim - 1], [0]))
    t = t.reshape([d for b in bases for d in (b, b)])  # (i_0, j_0, i_1, j_1, ...)
    rows = [2 * p for p in range(n)]
    cols = [2 * p + 1 for p in range(n - 1, -1, -1)]  # most significant column digit first
    N = int(np.prod(bases, dtype=np.int64))
    return t.transpose(rows + cols).reshape(N, N)


def dft_rows(N, rows, unreduced=False):
    """Rows of M(i, j) = v^(i j), v = exp(-2 pi i / N), with i j reduced modulo N exactly.

    unreduced=True forms exp(-2 pi i (i j) / N) from the unreduced product in FP64 instead, whose
    phase carries a rounding error of about 2 pi (i j / N) 2^-53."""
    idx = np.arange(N, dtype=np.int64)
    prod = np.outer(np.asarray(rows, dtype=np.int64), idx)
    if unreduced:
        return np.exp(-2j * np.pi * prod.astype(np.float64) / N)
    table = np.exp(-2j * np.pi * idx.astype(np.float64) / N)  # v^k, k = 0 .. N-1
    return table[prod % N]


def dft_matrix(N):
    return dft_rows(N, np.arange(N))


def distance(w, bases, unreduced=False, block=1024):
    """||M - T||_F / sqrt(N): the distance between the DFT matrix M and the Fourier TT T (rows of
    M formed block by block; unreduced as in dft_rows)."""
    N = int(np.prod(bases, dtype=np.int64))
    t = dense(w, bases)
    acc = 0.0
    for r0 in range(0, N, block):
        rows = np.arange(r0, min(N, r0 + block))
        dif = t[rows] - dft_rows(N, rows, unreduced)
        acc += float(np.sum(dif.real ** 2) + np.sum(dif.imag ** 2))
    return math.sqrt(acc) / math.sqrt(N)
