"""GPU parity of two large roundings against oracle scalars stored in tests/golden/.

The oracle needs minutes per train at these ranks, so tests/golden/make_large_rounding_scalars.py
ran it once and stored, per case, the ranks of round(y), ||y||, ||round(y)|| and the inner
products of round(y) and y with three fixed probe trains.  Two roundings whose relative
distance is e satisfy |<a, p> - <b, p>| <= e ||b|| ||p|| and | ||a|| - ||b|| | <= e ||b||, so
these scalars check the GPU result at the form's bar (1e-12 FP64, 1e-6 mixed) without the
oracle's cores.  Both cases run at the full bond ranks of their workloads (1792 after the 3D
Laplacian on a rank-256 train, 4096 for x (.) x at rank 64) with L = 24.
"""
import json
import math
import os

import numpy as np
import pytest
import torch

from paper_2602_20226_gb300 import inputs, qtt

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
L = 24


def _golden(case):
    with open(os.path.join(HERE, "golden", "large_rounding_scalars.json")) as f:
        g = json.load(f)
    assert g["L"] == L
    return g[case]


def _probes(tt):
    return [tt.TT.from_numpy(inputs.random_tt(900 + i, L, 2, 3)) for i in range(3)]


def _f64(tt, x):
    return tt.TT([c.double() for c in x.cores])


def _check_scalars(tt, Z, c, bar):
    z = _f64(tt, Z)
    nz = math.sqrt(tt.tt_inner(z, z))
    assert abs(nz - c["norm_z"]) <= bar * c["norm_z"], (nz, c["norm_z"])
    for p, ref in zip(_probes(tt), c["inner_z_p"]):
        np_ = math.sqrt(tt.tt_inner(p, p))
        assert abs(tt.tt_inner(z, p) - ref) <= bar * c["norm_z"] * np_, (tt.tt_inner(z, p), ref)


def test_laplacian3d_rank1792_mixed(cuda_lib):
    """3D Dirichlet Laplacian (rank 7) on a rank-256 FP32 train, mixed rounding at 1e-6: the
    ranks of the oracle, its norm and probe projections within 1e-6, and the rounding bound
    ||round(y) - y|| <= eps ||y|| (+ 1e-6 for the FP32 cores) on the GPU's own y."""
    tt = cuda_lib
    c = _golden("laplacian3d_r256")
    x = [a.astype(np.float32) for a in inputs.random_tt(31, L, 2, 256)]
    X = tt.TT.from_numpy(x, dtype=torch.float32)
    W = tt.MPO.from_numpy(qtt.laplacian_mpo(3, L // 3), dtype=torch.float32)
    Y = tt.tt_apply_mpo(W, X)
    assert Y.ranks == c["ranks_y"]
    Z, nrm = tt.tt_round(Y, c["eps"])
    assert Z.ranks == c["ranks_z"]
    assert abs(nrm - c["norm_y"]) <= 1e-6 * c["norm_y"]
    _check_scalars(tt, Z, c, 1e-6)
    zz, yy, zy = tt.tt_inner(Z, Z), tt.tt_inner(Y, Y), tt.tt_inner(Z, Y)
    e = math.sqrt(max(zz + yy - 2.0 * zy, 0.0) / yy)
    assert e <= c["eps"] + 1e-6, e


def test_hadamard_rank4096_fp64(cuda_lib):
    """x (.) x of a rank-64 train (bond ranks 4096), FP64 rounding at 1e-8: the oracle's ranks
    (at most r (r + 1) / 2 = 2080, the closed form), its norm and probe projections within
    1e-12."""
    tt = cuda_lib
    c = _golden("hadamard_r64")
    X = tt.TT.from_numpy(inputs.random_tt(32, L, 2, 64))
    Y = tt.tt_hadamard(X, X)
    assert Y.ranks == c["ranks_y"]
    Z, nrm = tt.tt_round(Y, c["eps"])
    assert Z.ranks == c["ranks_z"]
    assert max(Z.ranks) <= 64 * 65 // 2
    assert abs(nrm - c["norm_y"]) <= 1e-12 * c["norm_y"]
    _check_scalars(tt, Z, c, 1e-12)
