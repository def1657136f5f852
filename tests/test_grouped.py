"""Grouped-digit ("interleaved") layout on the host: every n_dims consecutive binary sites
merged into one core of mode 2^n_dims (Section 6, TrainShape mode 'interleaved').  The
library's grouped operators are pinned against the oracle's ungrouped operators as dense
matrices, and grouped trains against their ungrouped full tensors."""
import numpy as np
import pytest

from oracle import core, structured
from paper_2602_20226_gb300 import inputs, qtt


@pytest.mark.parametrize("n_dims,bits", [(1, 5), (2, 3), (3, 2)])
def test_grouped_laplacian_equals_the_oracle_operator(n_dims, bits):
    w = qtt.group_mpo_sites(qtt.laplacian_mpo(n_dims, bits), n_dims)
    assert [c.shape[1] for c in w] == [2 ** n_dims] * bits
    assert max(c.shape[3] for c in w) <= 2 * n_dims + 1
    ref = core.full_mpo(structured.laplacian_mpo(n_dims, bits))
    assert np.array_equal(core.full_mpo(w), ref)


def test_grouped_train_is_the_same_tensor():
    x = inputs.random_tt(11, 9, [2, 3, 2, 2, 5, 2, 2, 2, 3], 4)
    for g in (1, 3, 9):
        y = qtt.group_sites(x, g)
        assert len(y) == 9 // g
        assert np.abs(core.full(y).reshape(-1) - core.full(x).reshape(-1)).max() <= 1e-15


def test_group_size_must_divide():
    with pytest.raises(ValueError):
        qtt.group_sites(inputs.random_tt(1, 5, 2, 2), 2)
