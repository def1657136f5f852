"""GPU parity of apply + round on grouped-digit trains (mode 4 in 2D, 8 in 3D): the same
kernels as the binary layout, against the oracle on the same grouped cores."""
import numpy as np
import pytest
import torch

from oracle import core
from paper_2602_20226_gb300 import inputs, qtt

pytestmark = pytest.mark.gpu


def _e(a, b):
    return core.rel_err(a, b)


@pytest.mark.parametrize("n_dims,bits,rank", [(2, 8, 12), (3, 3, 6)])
def test_grouped_apply_round_fp64(cuda_lib, n_dims, bits, rank):
    tt = cuda_lib
    d = 2 ** n_dims
    x = inputs.random_tt(40 + n_dims, bits, d, rank)
    w = qtt.group_mpo_sites(qtt.laplacian_mpo(n_dims, bits), n_dims)
    Y = tt.tt_apply_mpo(tt.MPO.from_numpy(w), tt.TT.from_numpy(x))
    Z, _ = tt.tt_round(Y, 1e-10)
    ref = core.round_tt(core.apply_mpo(w, x), 1e-10)
    assert Z.ranks == core.ranks(ref)
    assert _e(Z.numpy(), ref) <= 1e-12


def test_grouped_apply_round_mixed(cuda_lib):
    tt = cuda_lib
    x = [c.astype(np.float32) for c in inputs.random_tt(45, 8, 4, 12)]
    w = qtt.group_mpo_sites(qtt.laplacian_mpo(2, 8), 2)
    Y = tt.tt_apply_mpo(tt.MPO.from_numpy(w, dtype=torch.float32), tt.TT.from_numpy(x, dtype=torch.float32))
    Z, _ = tt.tt_round(Y, 1e-6)
    ref = core.round_tt(core.apply_mpo(w, [c.astype(np.float64) for c in x]), 1e-6)
    assert Z.ranks == core.ranks(ref)
    assert _e(Z.numpy(), ref) <= 1e-6
