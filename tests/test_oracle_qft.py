"""Pins for the oracle's Fourier tensor train (Section 4.3).

* Every factor T_q is an MPO of rank b_q equal to v^(c_q i_q j) entry by entry.
* The exact product of the factors is numpy's FFT of the identity (a library routine that shares
  nothing with the construction): on the paper's mixed-radix example (N = 240, row bases
  3, 2, 2, 5, 2, 2 and the reversed bases for the columns) and on powers of two.
* At N = 2^13 the rounded products reproduce the distances the paper prints for the maximum ranks
  2, 4 and 8 (tests/golden/qft_distances_n8192.txt) to their two printed digits, the distance read
  as ||M - T||_F / sqrt(N).  At rank 16 the train is within 1e-12 of the exact DFT; the printed
  9.3e-11 is matched by the distance to a DFT matrix formed from the unreduced products i j in
  FP64 (whose own phase error is of that size).
"""
import os

import numpy as np
import pytest

from oracle import core, qft

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "qft_distances_n8192.txt")


def _golden():
    out = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                r, d = line.split()
                out[int(r)] = float(d)
    return out


@pytest.mark.parametrize("bases", [[3, 2, 2, 5, 2, 2], [2] * 6, [5, 3]])
def test_factor_mpos_are_rank_bq_phases(bases):
    n = len(bases)
    N = int(np.prod(bases))
    i = np.arange(N, dtype=np.int64)[:, None]
    j = np.arange(N, dtype=np.int64)[None, :]
    for q in range(n):
        f = qft.factor_mpo(bases, q)
        assert core.ranks(f) == [1] + [bases[q]] * (n - 1) + [1]
        cq = int(np.prod(bases[q + 1:]))
        iq = (i // cq) % bases[q]
        want = np.exp(-2j * np.pi * ((cq * iq * j) % N) / N)
        assert np.abs(qft.dense(f, bases) - want).max() <= 1e-14


@pytest.mark.parametrize("bases", [[3, 2, 2, 5, 2, 2], [2] * 8, [2, 3, 2]])
def test_exact_product_is_the_fft(bases):
    N = int(np.prod(bases))
    w = qft.fourier_mpo(bases)
    fft = np.fft.fft(np.eye(N), axis=0)  # column j is the transform of e_j: exp(-2 pi i i j / N)
    assert np.abs(qft.dense(w, bases) - fft).max() <= 1e-12
    # rounding without a rank cap keeps the matrix
    wr = qft.fourier_mpo(bases, eps=1e-14)
    assert np.abs(qft.dense(wr, bases) - fft).max() <= 1e-11


def test_paper_distances_n8192():
    bases = [2] * 13
    want = _golden()
    for r in (2, 4, 8):
        w = qft.fourier_mpo(bases, max_rank=r)
        assert max(core.ranks(w)) == r
        d = qft.distance(w, bases)
        assert float(f"{d:.1e}") == want[r], (r, d)
    w = qft.fourier_mpo(bases, max_rank=16)
    assert max(core.ranks(w)) == 16
    d = qft.distance(w, bases)
    assert d <= 1e-12, d
    d_raw = qft.distance(w, bases, unreduced=True)
    assert abs(d_raw / want[16] - 1.0) <= 0.1, d_raw
    assert d_raw >= 100 * d  # the unreduced matrix's own error, not the train's
