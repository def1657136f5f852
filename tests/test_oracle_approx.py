"""Pins for the oracle's approximate einsums (Section 3.2 decomposition / zip-up, Section 3.3
variational fit, Eq. (variational)) for y = W x.

* Without truncation every zip-up is exact (brute force on the full tensor), for every super-core
  size.  With the super-core spanning the whole train its norm is the result's and the steps are
  the truncated SVDs of the rounding: the same ranks as core.round_tt, the same tensor to 1e-12,
  error within eps ||y||.  Ranks never exceed max_rank.
* Every local update of the variational fit is the derivative of <C | y> with respect to the
  centre: checked against grad.inner_vjp (independent environment code).  With the other cores
  orthonormal that update is the exact minimiser over the centre, so ||C - y|| never increases
  (the whole trace is checked), a fit started from the rounding at rank r ends at least as close
  as the rounding, an exactly representable target is a fixed point, and the two-site fit
  recovers such a target from a random start.
"""
import numpy as np
import pytest

from oracle import approx, core, grad
from paper_2602_20226_gb300 import inputs

L = 10


def _problem():
    x = inputs.random_tt(3, L, 2, 6)
    w = inputs.random_mpo(4, L, 2, 3)
    return w, x, core.apply_mpo(w, x)


@pytest.mark.parametrize("ncores", [1, 2, 3, L])
def test_decomposition_exact_without_truncation(ncores):
    w, x, y = _problem()
    z = approx.decomposition_apply(w, x, 0.0, ncores=ncores)
    fy = core.full(y)
    assert np.linalg.norm(core.full(z) - fy) <= 1e-13 * np.linalg.norm(fy)


@pytest.mark.parametrize("eps", [1e-1, 1e-2])
def test_decomposition_over_the_whole_train_is_the_rounding(eps):
    w, x, y = _problem()
    z = approx.decomposition_apply(w, x, eps, ncores=L)
    ref = core.round_tt(y, eps)
    assert core.ranks(z) == core.ranks(ref)
    assert core.rel_err(z, ref) <= 1e-12
    fy = core.full(y)
    assert np.linalg.norm(core.full(z) - fy) <= eps * np.linalg.norm(fy)


@pytest.mark.parametrize("ncores", [1, 2])
def test_decomposition_rank_cap(ncores):
    w, x, _ = _problem()
    z = approx.decomposition_apply(w, x, 0.0, max_rank=5, ncores=ncores)
    assert max(core.ranks(z)) == 5


@pytest.mark.parametrize("ncores", [1, 2])
def test_variational_centre_is_the_overlap_gradient(ncores):
    """After a sweep the centre sits on site 1 and equals d<C|y>/dC_1 (the other cores being
    orthonormal), with and without a binding rank cap."""
    w, x, y = _problem()
    for r in (5, None):
        c0 = core.round_tt(y, 0.0, max_rank=r or 64)
        c = approx.variational_apply(w, x, c0, nsweeps=1, ncores=ncores, max_rank=r)
        g, _ = grad.inner_vjp(c, y)
        assert np.abs(c[0] - g[0]).max() <= 1e-12 * np.abs(g[0]).max()


@pytest.mark.parametrize("ncores", [1, 2])
@pytest.mark.parametrize("r", [4, 8])
def test_variational_updates_never_increase_the_distance(ncores, r):
    w, x, y = _problem()
    c0 = core.round_tt(y, 0.0, max_rank=r)
    start = core.norm(core.add(c0, core.scale(y, -1.0)))
    trace = []
    c = approx.variational_apply(w, x, c0, nsweeps=2, ncores=ncores, max_rank=r, trace=trace)
    assert max(core.ranks(c)) == r
    seq = [start] + trace
    assert all(b <= a * (1 + 1e-12) for a, b in zip(seq, seq[1:])), seq
    assert trace[-1] <= start


@pytest.mark.parametrize("ncores", [1, 2])
def test_variational_exact_target_is_a_fixed_point(ncores):
    w, x, y = _problem()
    c0 = core.round_tt(y, 1e-14)
    c = approx.variational_apply(w, x, c0, nsweeps=1, ncores=ncores)
    assert core.rel_err(c, y) <= 1e-12


def test_variational_two_site_recovers_target_from_random_start():
    w, x, y = _problem()
    c0 = inputs.random_tt(9, L, 2, 4)
    c = approx.variational_apply(w, x, c0, nsweeps=2, ncores=2, eps=1e-13)
    assert core.rel_err(c, y) <= 1e-12
    assert core.ranks(c) == core.ranks(core.round_tt(y, 1e-12))
