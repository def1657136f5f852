"""Nominal work of one apply + round, by a fixed counting convention.

The convention (used for every arithmetic form, so forms compare on equal work):
    GEMM (m x k) (k x n)             2 m n k
    Householder QR + thin Q, m >= n  4 m n^2 - 4 n^3 / 3
    SVD of an n x n factor           12 n^3
    apply                            2 a a' r r' d^2 per core
    hadamard                         1 per output element
    eval                             2 sum_k r_{k-1} r_k per sample
The rounding count follows the two sweeps exactly as they run: the right-to-left
LQ of every core of the input and the R-multiply into its left neighbour, then for
every bond the QR (or LQ for a wide core), the SVD of the square factor and the three
GEMMs that form the truncated cores.
"""
from __future__ import annotations


def qr_flops(m: int, n: int) -> float:
    if m < n:
        m, n = n, m
    return 4.0 * m * n * n - 4.0 * n ** 3 / 3.0


def apply_flops(w_ranks, x_ranks, dims) -> float:
    return sum(2.0 * w_ranks[k] * w_ranks[k + 1] * x_ranks[k] * x_ranks[k + 1] * dims[k] ** 2
               for k in range(len(dims)))


def hadamard_flops(x_ranks, y_ranks, dims) -> float:
    return float(sum(x_ranks[k] * y_ranks[k] * dims[k] * x_ranks[k + 1] * y_ranks[k + 1]
                     for k in range(len(dims))))


def eval_flops(ranks, n_samples: int) -> float:
    return 2.0 * n_samples * sum(ranks[k] * ranks[k + 1] for k in range(len(ranks) - 1))


def round_flops(in_ranks, out_ranks, dims) -> dict:
    """Nominal flops of tt_round given the input and output ranks."""
    L = len(dims)
    r = list(in_ranks)
    qr = svd = gemm = 0.0
    # right-to-left: LQ of C_k (r_{k-1} x d r_k), C_{k-1} <- C_{k-1} L
    for k in range(L - 1, 0, -1):
        m, n = dims[k] * r[k + 1], r[k]
        p = min(m, n)
        qr += qr_flops(m, n)
        gemm += 2.0 * r[k - 1] * dims[k - 1] * p * n
        r[k] = p
    # left-to-right: QR or LQ, SVD of the p x p factor, three GEMMs
    for k in range(L - 1):
        m, n = r[k] * dims[k], r[k + 1]
        p = min(m, n)
        rn = out_ranks[k + 1]
        qr += qr_flops(m, n)
        svd += 12.0 * p ** 3
        if m >= n:
            gemm += 2.0 * m * rn * p + 2.0 * rn * n * p
        else:
            gemm += 2.0 * rn * n * m
        gemm += 2.0 * rn * dims[k + 1] * r[k + 2] * n
        r[k] = out_ranks[k]
        r[k + 1] = rn
    return {"qr": qr, "svd": svd, "gemm": gemm, "total": qr + svd + gemm}
