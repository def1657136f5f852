"""Host-side constructors of structured quantics TTs and MPOs (Section 4).

These build the inputs the library's kernels consume: the Dirichlet Laplacian MPO
on an interleaved binary layout (from the shift decomposition of Section 4.2) and
the closed-form exp / cos / sin TTs of Section 4.1.  Pure numpy, host memory; the
caller moves the cores to the device (``TT.from_numpy`` / ``MPO.from_numpy``).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["laplacian_mpo", "second_difference_mpo", "exp_tt", "cos_tt", "sin_tt",
           "interleave_sites", "group_sites", "group_mpo_sites"]

_I = np.eye(2)
_J = np.array([[0.0, 0.0], [1.0, 0.0]])  # shift by +1 within one binary digit: J[1][0] = 1
_JT = _J.T


def interleave_sites(n_dims: int, bits: int) -> list[int]:
    """Owner dimension of each site for the layout x_1, y_1, (z_1,) x_2, y_2, ..."""
    return [k % n_dims for k in range(n_dims * bits)]


def laplacian_mpo(n_dims: int, bits: int) -> list[np.ndarray]:
    """Dirichlet Laplacian sum_t (S_t^+ + S_t^- - 2 I) on n_dims interleaved binary dims.

    Each one-dimension second difference is a sum of the +1 shift, the -1 shift and
    -2 I; every shift carries a borrow from the least significant digit upwards (the
    rank-2 structure of Eq. (shif_dec) in base 2).  The bond states alive between
    sites k and k+1 are enumerated directly:
      'pend'      no term chosen yet (alive while some dimension still has sites ahead),
      (t, '+')    dimension t's +1 shift has been chosen and its carry propagates,
      (t, '-')    the same for the -1 shift,
      'done'      a term finished at its last digit (alive once any dimension has ended).
    Bond ranks are at most 2 n_dims + 1 (3 in 1D, 5 in 2D, 7 in 3D).
    """
    owner = interleave_sites(n_dims, bits)
    L = len(owner)
    first = {t: min(k for k in range(L) if owner[k] == t) for t in range(n_dims)}
    last = {t: max(k for k in range(L) if owner[k] == t) for t in range(n_dims)}

    def bond_states(b: int) -> list:
        """States alive on the bond right of site b - 1 (b = 0 .. L)."""
        if b == 0:
            return ["pend"]
        if b == L:
            return ["done"]
        st = []
        if any(last[t] >= b for t in range(n_dims)):
            st.append("pend")
        for t in range(n_dims):
            if first[t] < b <= last[t]:
                st += [(t, "+"), (t, "-")]
        if any(last[t] < b for t in range(n_dims)):
            st.append("done")
        return st

    cores = []
    for k in range(L):
        left, right = bond_states(k), bond_states(k + 1)
        li = {s: i for i, s in enumerate(left)}
        ri = {s: i for i, s in enumerate(right)}
        c = np.zeros((len(left), 2, 2, len(right)))
        t = owner[k]

        def put(a, b, m):
            if a in li and b in ri:
                c[li[a], :, :, ri[b]] += m

        # states of other dimensions pass through unchanged
        for s in left:
            if isinstance(s, tuple) and s[0] != t:
                put(s, s, _I)
        put("done", "done", _I)
        if k < last[t]:
            put("pend", "pend", _I)
            put("pend", (t, "+"), _J)
            put("pend", (t, "-"), _JT)
            put((t, "+"), (t, "+"), _JT)
            put((t, "-"), (t, "-"), _J)
        else:
            put("pend", "pend", _I)  # kept only if another dimension is still pending
            put("pend", "done", _J + _JT - 2.0 * _I)
            put((t, "+"), "done", _JT)
            put((t, "-"), "done", _J)
        cores.append(c)
    return cores


def second_difference_mpo(bits: int) -> list[np.ndarray]:
    """One-dimension Dirichlet second difference (rank 3)."""
    return laplacian_mpo(1, bits)


def _digit_steps(bits: int, lower: float, upper: float) -> list[np.ndarray]:
    h = (upper - lower) / (2 ** bits - 1)
    return [h * 2 ** (bits - 1 - q) * np.arange(2.0) for q in range(bits)]


def exp_tt(bits: int, lower: float, upper: float, v: float, x0: float = 0.0) -> list[np.ndarray]:
    """e^{v (x - x0)} on the uniform binary grid: rank 1 (Section 4.1, Eq. (exp_dec))."""
    steps = _digit_steps(bits, lower, upper)
    cores = [np.exp(v * s).reshape(1, 2, 1) for s in steps]
    cores[0] = cores[0] * math.exp(v * (lower - x0))
    return cores


def cos_tt(bits: int, lower: float, upper: float, v: float, x0: float = 0.0,
           phase: float = 0.0) -> list[np.ndarray]:
    """cos(v (x - x0) + phase) as the real rank-2 rotation TT (Section 4.1)."""
    steps = _digit_steps(bits, lower, upper)
    shift = (v * (lower - x0) + phase) / bits
    rots = []
    for s in steps:
        ang = v * s + shift
        ca, sa = np.cos(ang), np.sin(ang)
        rots.append(np.stack([np.stack([ca, -sa], axis=-1), np.stack([sa, ca], axis=-1)], axis=0))
    if bits == 1:
        return [(0.5 * rots[0].sum(axis=(0, 2))).reshape(1, 2, 1)]
    cores = list(rots)
    cores[0] = (0.5 * rots[0].sum(axis=0)).reshape(1, 2, 2)
    cores[-1] = rots[-1].sum(axis=2).reshape(2, 2, 1)
    return cores


def sin_tt(bits: int, lower: float, upper: float, v: float, x0: float = 0.0) -> list[np.ndarray]:
    """sin(v (x - x0)) as the rotation TT shifted by pi/2."""
    return cos_tt(bits, lower, upper, v, x0, phase=-0.5 * math.pi)


def group_sites(cores: list[np.ndarray], g: int) -> list[np.ndarray]:
    """The same tensor with every g consecutive sites merged into one core of mode d^g: the
    grouped ("interleaved") layout that puts the digits (x_q, y_q[, z_q]) of one scale on a
    single core (Section 6, TrainShape mode 'interleaved'; d = 4 in 2D, 8 in 3D).  The
    merged index keeps the first site's digit most significant, i = i_1 d_2 + i_2, as the
    quantics order of Eq. (quantization).  len(cores) must be a multiple of g."""
    if g < 1 or len(cores) % g:
        raise ValueError("the number of sites must be a multiple of the group size")
    out = []
    for k in range(0, len(cores), g):
        c = cores[k]
        for nxt in cores[k + 1:k + g]:
            r0, d1, _ = c.shape
            _, d2, r2 = nxt.shape
            c = np.tensordot(c, nxt, axes=([2], [0])).reshape(r0, d1 * d2, r2)
        out.append(np.ascontiguousarray(c))
    return out


def group_mpo_sites(cores: list[np.ndarray], g: int) -> list[np.ndarray]:
    """group_sites for an MPO: cores W[a, i, j, a'] merged g at a time into
    W[a, (i_1 .. i_g), (j_1 .. j_g), a'] (output and input digits each first-site major)."""
    if g < 1 or len(cores) % g:
        raise ValueError("the number of sites must be a multiple of the group size")
    out = []
    for k in range(0, len(cores), g):
        c = cores[k]
        for nxt in cores[k + 1:k + g]:
            a0, do1, di1, _ = c.shape
            _, do2, di2, a2 = nxt.shape
            t = np.tensordot(c, nxt, axes=([3], [0]))  # a0, do1, di1, do2, di2, a2
            c = t.transpose(0, 1, 3, 2, 4, 5).reshape(a0, do1 * do2, di1 * di2, a2)
        out.append(np.ascontiguousarray(c))
    return out
