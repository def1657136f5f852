"""GPU parity of the rounding adjoint (tt_round_backward, FP64 form) against the oracle.

The loss is <round(x), y> for a fixed train y (a function of the represented tensor, so the
gradient does not depend on either side's gauge): each side forms the cotangent of its own
output cores with its own inner-product adjoint and runs its own rounding adjoint; the
gradients w.r.t. the cores of x must agree.  The oracle's adjoint is pinned by central
differences and by the closed form (no truncation: the gradient of <x, y>).

Bar.  Both sides are FP64 but factor the cores differently (LAPACK vs the library's QR and
Jacobi), so they differ by the response of the gradient to O(1e-15) relative changes of the
factors.  That response depends on the input: the adjoint of a truncated SVD divides by the
gaps between kept and dropped singular values, and with a dropped part at 1e-6 of the kept
one a 1e-15 relative perturbation of x moves the oracle's own gradient by ~1e-10 of its
largest entry (at 1e-3: ~3e-14).  Each case therefore measures that response of the oracle
(x perturbed by 1e-15 relative noise) and allows 30 times it, with 1e-11 of the largest
entry as the floor.
"""
import numpy as np
import pytest

from oracle import core, grad
from paper_2602_20226_gb300 import _abi, inputs

pytestmark = pytest.mark.gpu


def _gap_train(seed, L, r_big, r_small, scale):
    """big + scale * small, re-expressed without redundant bonds (the oracle's rounding at
    1e-14 keeps the tensor), so every bond rank equals the rank of its unfolding."""
    caps = [min(2 ** k, 2 ** (L - k)) for k in range(L + 1)]
    big = inputs.random_tt(seed, L, 2, [min(r_big, c) for c in caps])
    small = inputs.random_tt(seed + 1, L, 2, [min(r_small, c) for c in caps])
    x = core.round_tt(core.add(big, core.scale(small, scale)), 1e-14)
    assert all(r <= c for r, c in zip(core.ranks(x), caps))
    return x


def _gpu_grad(tt, x, y, eps):
    X = tt.TT.from_numpy(x)
    Y = tt.TT.from_numpy(y)
    Z, _ = tt.tt_round(X, eps)
    dZ, _ = tt.tt_inner_backward(Z, Y, 1.0, want_y=False)
    dX = tt.tt_round_backward(X, eps, dZ)
    return [c.cpu().numpy() for c in dX.cores], Z.ranks


def _oracle_grad(x, y, eps):
    out = core.round_tt(x, eps)
    dout, _ = grad.inner_vjp(out, y)
    return grad.round_vjp(x, eps, dout), core.ranks(out)


def _dev(a, b):
    """Largest deviation of a from b, relative to the largest entry of b."""
    scale = max(np.abs(v).max() for v in b)
    return max(np.abs(u - v).max() for u, v in zip(a, b)) / scale


def _close(a, b, tol):
    return _dev(a, b) <= tol


def _oracle_response(x, y, eps, ref, seed=7):
    """The oracle gradient's change under a 1e-15 relative perturbation of the cores of x."""
    rng = np.random.default_rng(seed)
    xp = [c * (1.0 + 1e-15 * rng.standard_normal(c.shape)) for c in x]
    return _dev(_oracle_grad(xp, y, eps)[0], ref)


def test_round_backward_without_truncation(cuda_lib):
    """eps below every singular value: the gradient of <round(x), y> is that of <x, y>."""
    x = _gap_train(501, 9, 6, 3, 1e-2)
    y = inputs.random_tt(503, 9, 2, 4)
    got, ranks = _gpu_grad(cuda_lib, x, y, 1e-13)
    assert ranks == core.ranks(x)
    ref, _ = grad.inner_vjp(x, y)
    assert _close(got, ref, 1e-10)


@pytest.mark.parametrize("gap,eps", [(1e-6, 1e-4), (1e-6, 1e-9), (1e-3, 1e-2)])
def test_round_backward_matches_oracle(cuda_lib, gap, eps):
    """x = big + gap * small.  (1e-6, 1e-4) truncates the small part (SVD bonds); (1e-6, 1e-9)
    keeps it (bonds certified full rank: QR adjoints); (1e-3, 1e-2) truncates the small part
    and cuts into the big one at some bonds."""
    L = 12
    x = _gap_train(511, L, 12, 4, gap)
    y = inputs.random_tt(513, L, 2, 5)
    got, ranks = _gpu_grad(cuda_lib, x, y, eps)
    ref, oranks = _oracle_grad(x, y, eps)
    assert ranks == oranks
    bar = max(1e-11, 30.0 * _oracle_response(x, y, eps, ref))
    dev = _dev(got, ref)
    assert dev <= bar, (dev, bar)


def test_round_backward_heavy_truncation(cuda_lib):
    """A short train whose middle bond is cut from 8 to 4 (and its neighbours with it)."""
    x = _gap_train(521, 6, 40, 3, 1e-5)
    y = inputs.random_tt(523, 6, 2, 3)
    got, ranks = _gpu_grad(cuda_lib, x, y, 1e-3)
    ref, oranks = _oracle_grad(x, y, 1e-3)
    assert ranks == oranks
    assert _close(got, ref, 1e-10)


def test_round_backward_singular_factor_rejected(cuda_lib):
    """Two equal rows in core 3 make the right-to-left factor R_3 singular (the bond rank r_2
    exceeds the rank of the right unfolding at that bond): the thin-QR adjoint needs R_3^-1,
    so there is no derivative and the call reports TT_ERR_NUMERIC.  (Redundancy on the left
    of a bond does not do this: the right-to-left sweep never factors the left part, and a
    wide factor is handled by its own QR adjoint.)"""
    tt = cuda_lib
    x = inputs.random_tt(531, 6, 2, 4)
    x[3][1] = x[3][0]
    X = tt.TT.from_numpy(x)
    Z, _ = tt.tt_round(X, 1e-10)
    dZ, _ = tt.tt_inner_backward(Z, tt.TT.from_numpy(inputs.random_tt(532, 6, 2, 2)), 1.0, want_y=False)
    with pytest.raises(tt.TTError) as ei:
        tt.tt_round_backward(X, 1e-10, dZ)
    assert ei.value.code == _abi.TT_ERR_NUMERIC
