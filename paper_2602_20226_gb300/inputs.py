"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle.

This module only draws random numbers and lays them out; it contains none of the
tensor-train arithmetic (no contraction, orthogonalisation, truncation or operator
construction).  Every array is produced on the host in float64 from a numpy PCG64
stream, so the CUDA path and the oracle see bit-identical inputs.

Conventions (Section 2, Eq. (quantization) and Eq. (vector_dec)):
  * a TT of length L is a list of cores G_k with shape (r_{k-1}, d_k, r_k),
    r_0 = r_L = 1, stored row-major;
  * an MPO is a list of cores W_k with shape (a_{k-1}, d_k(out), d_k(in), a_k);
  * site 1 carries the most significant digit.

Random TTs follow the recipe "cores i.i.d. N(0,1), normalised": core k is drawn
N(0,1) and scaled by 1/sqrt(d_k * r_k), which makes E||x||^2 = 1 for any length.
Interior ranks are the nominal rank everywhere (not capped at d^k), so rounding
really has to reduce the edge bonds.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "rng",
    "random_tt",
    "random_mpo",
    "random_digits",
    "tt_ranks",
    "batch_shapes",
    "fit_targets",
]


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def tt_ranks(L: int, r: int) -> list[int]:
    """Uncapped nominal ranks [1, r, r, ..., r, 1]."""
    if L < 1:
        raise ValueError("L must be >= 1")
    return [1] + [int(r)] * (L - 1) + [1]


def random_tt(seed: int, L: int, d: int | list[int], r: int | list[int],
              dtype=np.float64) -> list[np.ndarray]:
    """Seeded Gaussian TT, core k ~ N(0,1)/sqrt(d_k r_k)."""
    g = rng(seed)
    ds = [int(d)] * L if np.isscalar(d) else [int(v) for v in d]
    ranks = tt_ranks(L, r) if np.isscalar(r) else [int(v) for v in r]
    if len(ds) != L or len(ranks) != L + 1 or ranks[0] != 1 or ranks[-1] != 1:
        raise ValueError("bad TT shape")
    cores = []
    for k in range(L):
        c = g.standard_normal((ranks[k], ds[k], ranks[k + 1]))
        c *= 1.0 / np.sqrt(ds[k] * ranks[k + 1])
        cores.append(np.ascontiguousarray(c.astype(dtype)))
    return cores


def random_mpo(seed: int, L: int, d: int, a: int, dtype=np.float64) -> list[np.ndarray]:
    """Seeded Gaussian MPO with uncapped bond a, core k ~ N(0,1)/sqrt(d a_k)."""
    g = rng(seed)
    ranks = tt_ranks(L, a)
    cores = []
    for k in range(L):
        c = g.standard_normal((ranks[k], d, d, ranks[k + 1]))
        c *= 1.0 / np.sqrt(d * ranks[k + 1])
        cores.append(np.ascontiguousarray(c.astype(dtype)))
    return cores


def random_digits(seed: int, n: int, d: list[int]) -> np.ndarray:
    """n index tuples drawn uniformly: digit k uniform in [0, d_k).  uint8 [n, L].

    Drawing each digit uniformly is the same as drawing the flat index uniformly,
    because the digit map of Eq. (quantization) is a bijection.
    """
    g = rng(seed)
    L = len(d)
    out = np.empty((n, L), dtype=np.uint8)
    for k in range(L):
        out[:, k] = g.integers(0, int(d[k]), size=n, dtype=np.uint8)
    return out


def batch_shapes(seed: int, n_tt: int, L_range=(20, 60), r_range=(8, 128),
                 a_choices=(3, 4, 5)) -> list[tuple[int, int, int]]:
    """(L, r, a) per TT for an uneven batch: L and r integer-uniform (inclusive)."""
    g = rng(seed)
    out = []
    for _ in range(n_tt):
        L = int(g.integers(L_range[0], L_range[1] + 1))
        r = int(g.integers(r_range[0], r_range[1] + 1))
        a = int(g.choice(np.asarray(a_choices)))
        out.append((L, r, a))
    return out


def fit_targets(digits: np.ndarray, bits: int, dims: int = 2,
                lower: float = -1.0, upper: float = 1.0) -> np.ndarray:
    """Sample targets f(x, y) = exp(-(x^2 + y^2)) cos(8x) for interleaved binary digits.

    Data recipe for the fitting workload: site q*dims + t holds bit q (most
    significant first) of coordinate t; the grid is x(i) = lower + (upper-lower) i/(2^bits - 1).
    """
    n = digits.shape[0]
    coords = []
    for t in range(dims):
        idx = np.zeros(n, dtype=np.int64)
        for q in range(bits):
            idx = idx * 2 + digits[:, q * dims + t].astype(np.int64)
        coords.append(lower + (upper - lower) * idx.astype(np.float64) / float(2 ** bits - 1))
    x, y = coords[0], coords[1]
    return np.exp(-(x * x + y * y)) * np.cos(8.0 * x)
