"""GPU parity of the exact core-by-core operations and their adjoints.

Every check runs the CUDA path through the C ABI and the FP64 oracle on the same
seeded inputs and compares element by element.

Tolerances (FP64 cores): apply and hadamard sum at most d products per element,
so they agree to a few ulp: |gpu - oracle| <= 1e-13 |oracle| + 1e-15 max|oracle|.
inner/eval/gradients contract whole trains in a different order than the oracle;
the bound used is 1e-12 of the natural scale (||x|| ||y|| for inner, the RMS of the
values for eval, the largest gradient entry for gradients).
FP32 cores: the oracle runs on the same FP32 values in FP64; the bound is 1e-5 of
the scale (a few FP32 ulps accumulated over the train).
"""
import numpy as np
import pytest
import torch

from oracle import core, grad
from paper_2602_20226_gb300 import inputs, qtt

pytestmark = pytest.mark.gpu


def _tt(seed, L, r, d=2):
    return inputs.random_tt(seed, L, d, r)


def _close(gpu, ref, rtol, atol_scale):
    ref = np.asarray(ref)
    gpu = np.asarray(gpu)
    scale = np.abs(ref).max() if ref.size else 0.0
    return np.all(np.abs(gpu - ref) <= rtol * np.abs(ref) + atol_scale * scale)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("case", ["c1", "ragged", "modes", "single"])
def test_apply_mpo_parity(cuda_lib, dtype, case):
    tt = cuda_lib
    if case == "c1":
        x = _tt(1, 10, 8)
        w = qtt.second_difference_mpo(10)
    elif case == "ragged":
        x = inputs.random_tt(2, 7, 2, [1, 3, 17, 33, 5, 9, 2, 1])
        w = inputs.random_mpo(3, 7, 2, 4)
    elif case == "modes":
        x = inputs.random_tt(4, 5, [2, 3, 5, 2, 7], [1, 4, 6, 6, 3, 1])
        g = inputs.rng(5)
        ar = [1, 3, 2, 4, 2, 1]
        dd = [2, 3, 5, 2, 7]
        w = [g.standard_normal((ar[k], dd[k], dd[k], ar[k + 1])) for k in range(5)]
    else:
        x = inputs.random_tt(6, 1, 4, [1, 1])
        w = [inputs.rng(7).standard_normal((1, 4, 4, 1))]
    if dtype == torch.float32:
        x = [c.astype(np.float32).astype(np.float64) for c in x]
        w = [c.astype(np.float32).astype(np.float64) for c in w]
    X = tt.TT.from_numpy(x, dtype=dtype)
    Wd = tt.MPO.from_numpy(w, dtype=dtype)
    Y = tt.tt_apply_mpo(Wd, X)
    ref = core.apply_mpo(w, x)
    assert Y.ranks == core.ranks(ref)
    rtol, at = (1e-13, 1e-15) if dtype == torch.float64 else (1e-5, 1e-6)
    for a, b in zip(Y.numpy(), ref):
        assert a.shape == b.shape
        assert _close(a, b, rtol, at)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("case", ["square", "ragged", "modes"])
def test_hadamard_parity(cuda_lib, dtype, case):
    tt = cuda_lib
    if case == "square":
        x = _tt(10, 12, 16)
        y = x
    elif case == "ragged":
        x = inputs.random_tt(11, 6, 2, [1, 5, 33, 7, 2, 3, 1])
        y = inputs.random_tt(12, 6, 2, [1, 3, 2, 40, 9, 1, 1])
    else:
        x = inputs.random_tt(13, 4, [3, 2, 5, 2], [1, 4, 3, 2, 1])
        y = inputs.random_tt(14, 4, [3, 2, 5, 2], [1, 2, 5, 3, 1])
    if dtype == torch.float32:
        x = [c.astype(np.float32).astype(np.float64) for c in x]
        y = [c.astype(np.float32).astype(np.float64) for c in y]
    Z = tt.tt_hadamard(tt.TT.from_numpy(x, dtype=dtype), tt.TT.from_numpy(y, dtype=dtype))
    ref = core.hadamard(x, y)
    assert Z.ranks == core.ranks(ref)
    rtol, at = (1e-13, 1e-15) if dtype == torch.float64 else (1e-6, 1e-7)
    for a, b in zip(Z.numpy(), ref):
        assert _close(a, b, rtol, at)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_inner_parity(cuda_lib, dtype):
    tt = cuda_lib
    for seed, (L, rx, ry) in enumerate([(10, 8, 8), (40, 64, 16), (7, 33, 5), (1, 1, 1)]):
        x = _tt(20 + seed, L, rx)
        y = _tt(40 + seed, L, ry)
        if dtype == torch.float32:
            x = [c.astype(np.float32).astype(np.float64) for c in x]
            y = [c.astype(np.float32).astype(np.float64) for c in y]
        v = tt.tt_inner(tt.TT.from_numpy(x, dtype=dtype), tt.TT.from_numpy(y, dtype=dtype))
        ref = core.inner(x, y)
        scale = core.norm(x) * core.norm(y)
        tol = 1e-12 if dtype == torch.float64 else 1e-12  # FP64 environments in both dtypes
        assert abs(v - ref) <= tol * scale, (L, v, ref)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("case", [(10, 8, 2, 1000), (40, 64, 2, 5000), (7, 37, 3, 2000), (6, 130, 3, 777), (3, 2, 5, 0)])
def test_eval_parity(cuda_lib, dtype, case):
    tt = cuda_lib
    L, r, d, n = case
    x = _tt(60 + L, L, r, d)
    if dtype == torch.float32:
        x = [c.astype(np.float32).astype(np.float64) for c in x]
    dg = inputs.random_digits(61, n, [d] * L)
    v = tt.tt_eval(tt.TT.from_numpy(x, dtype=dtype), torch.as_tensor(dg, device="cuda"))
    ref = core.evaluate(x, dg) if n else np.zeros(0)
    got = v.cpu().double().numpy()
    assert got.shape == (n,)
    if n:
        rms = np.sqrt(np.mean(ref ** 2))
        tol = 1e-12 if dtype == torch.float64 else 1e-5
        assert np.max(np.abs(got - ref)) <= tol * rms * max(1.0, L / 10)


def test_apply_backward_parity(cuda_lib):
    tt = cuda_lib
    x = inputs.random_tt(70, 6, 2, [1, 3, 5, 4, 6, 2, 1])
    w = inputs.random_mpo(71, 6, 2, 3)
    y = core.apply_mpo(w, x)
    dy = [inputs.rng(72 + k).standard_normal(c.shape) for k, c in enumerate(y)]
    gx, gw = tt.tt_apply_mpo_backward(tt.MPO.from_numpy(w), tt.TT.from_numpy(x), tt.TT.from_numpy(dy))
    rx, rw = grad.apply_mpo_vjp(w, x, dy)
    for a, b in zip(gx.numpy(), rx):
        assert _close(a, b, 1e-12, 1e-14)
    for a, b in zip(gw.numpy(), rw):
        assert _close(a, b, 1e-12, 1e-14)


def test_hadamard_backward_parity(cuda_lib):
    tt = cuda_lib
    x = inputs.random_tt(80, 5, 2, [1, 3, 4, 2, 5, 1])
    y = inputs.random_tt(81, 5, 2, [1, 2, 6, 3, 2, 1])
    z = core.hadamard(x, y)
    dz = [inputs.rng(82 + k).standard_normal(c.shape) for k, c in enumerate(z)]
    gx, gy = tt.tt_hadamard_backward(tt.TT.from_numpy(x), tt.TT.from_numpy(y), tt.TT.from_numpy(dz))
    rx, ry = grad.hadamard_vjp(x, y, dz)
    for a, b in zip(gx.numpy(), rx):
        assert _close(a, b, 1e-12, 1e-14)
    for a, b in zip(gy.numpy(), ry):
        assert _close(a, b, 1e-12, 1e-14)


def test_inner_backward_parity(cuda_lib):
    tt = cuda_lib
    x = _tt(90, 12, 9)
    y = _tt(91, 12, 5)
    gx, gy = tt.tt_inner_backward(tt.TT.from_numpy(x), tt.TT.from_numpy(y), 1.5)
    rx, ry = grad.inner_vjp(x, y, 1.5)
    for a, b in zip(gx.numpy(), rx):
        assert _close(a, b, 1e-11, 1e-13)
    for a, b in zip(gy.numpy(), ry):
        assert _close(a, b, 1e-11, 1e-13)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_eval_backward_tiles_and_modes(cuda_lib, dtype):
    """Ranks above one 64 x 64 accumulation tile (bond 80), mixed modes d in {2, 3, 5} (digit
    groups of the accumulation), out-of-order digits and a ragged sample count.  FP32 cores
    are rounded first, so both sides evaluate the same tensor; the FP32 bound allows FP32
    states and slice sums (~1e-6 relative)."""
    tt = cuda_lib
    modes = [3, 2, 5, 2, 3, 2]
    ranks = [1, 3, 6, 30, 80, 6, 2, 1][:len(modes) + 1]
    ranks[-1] = 1
    x = inputs.random_tt(120, len(modes), modes, ranks)
    if dtype == torch.float32:
        x = [c.astype(np.float32).astype(np.float64) for c in x]
    n = 4099
    dg = inputs.random_digits(121, n, modes)
    w = inputs.rng(122).standard_normal(n)
    g = tt.tt_eval_backward(tt.TT.from_numpy(x, dtype=dtype), torch.as_tensor(dg, device="cuda"),
                            torch.as_tensor(w, device="cuda"))
    ref = grad.evaluate_vjp(x, dg, w)
    scale = max(np.abs(b).max() for b in ref)
    tol = 1e-12 if dtype == torch.float64 else 2e-5
    for a, b in zip(g.numpy(), ref):
        assert np.abs(a.astype(np.float64) - b).max() <= tol * scale


@pytest.mark.parametrize("n", [1, 300, 20000])
def test_eval_backward_parity(cuda_lib, n):
    tt = cuda_lib
    L = 8
    x = _tt(100, L, 6)
    dg = inputs.random_digits(101, n, [2] * L)
    w = inputs.rng(102).standard_normal(n)
    g = tt.tt_eval_backward(tt.TT.from_numpy(x), torch.as_tensor(dg, device="cuda"),
                            torch.as_tensor(w, device="cuda"))
    ref = grad.evaluate_vjp(x, dg, w)
    for a, b in zip(g.numpy(), ref):
        assert _close(a, b, 1e-11, 1e-13)
