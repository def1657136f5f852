"""Gradients through the autograd wrappers against the oracle's adjoints.

The oracle's adjoints are pinned to FP64 central finite differences (test_oracle_grad);
here the GPU gradients (FP64 cores) must match them to 1e-10 of the largest gradient
entry (the adjoint sweeps reorder the sums), and FP32 cores to 1e-4.  The evaluation
workload at full size (2^20 samples, L = 40, rank 64, FP32) is checked on a sample of
outputs the oracle evaluates one by one.
"""
import numpy as np
import pytest
import torch

from oracle import core, grad, structured
from paper_2602_20226_gb300 import inputs, qtt
from paper_2602_20226_gb300.autograd import tt_apply_ad, tt_eval_ad, tt_hadamard_ad, tt_inner_ad

pytestmark = pytest.mark.gpu


def _params(cores, dtype=torch.float64):
    return [torch.tensor(c, dtype=dtype, device="cuda", requires_grad=True) for c in cores]


def _close(gpu, ref, tol):
    scale = max(np.abs(r).max() for r in ref)
    return all(np.abs(g.detach().double().cpu().numpy() - r).max() <= tol * scale for g, r in zip(gpu, ref))


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-10), (torch.float32, 1e-4)])
def test_fit_loss_gradient(cuda_lib, dtype, tol):
    bits = 6
    L = 2 * bits
    x = inputs.random_tt(200, L, 2, 8)
    if dtype == torch.float32:
        x = [c.astype(np.float32).astype(np.float64) for c in x]
    dg = inputs.random_digits(201, 5000, [2] * L)
    f = inputs.fit_targets(dg, bits)
    xs = _params(x, dtype)
    d = torch.as_tensor(dg, device="cuda")
    ft = torch.as_tensor(f, dtype=dtype, device="cuda")
    loss = 0.5 * ((tt_eval_ad(xs, d) - ft) ** 2).mean()
    loss.backward()
    ref = grad.fit_loss_grad(x, dg, f)
    lv = float(loss.detach())
    assert abs(lv - grad.fit_loss(x, dg, f)) <= (1e-12 if dtype == torch.float64 else 1e-5) * lv
    assert _close([p.grad for p in xs], ref, tol)


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-10), (torch.float32, 1e-4)])
def test_residual_gradient(cuda_lib, dtype, tol):
    bits = 4
    L = 2 * bits
    w = qtt.laplacian_mpo(2, bits)
    x = inputs.random_tt(210, L, 2, 4)
    b = inputs.random_tt(211, L, 2, 3)
    if dtype == torch.float32:
        x = [c.astype(np.float32).astype(np.float64) for c in x]
        b = [c.astype(np.float32).astype(np.float64) for c in b]
    ws = [torch.tensor(c, dtype=dtype, device="cuda") for c in w]
    xs = _params(x, dtype)
    bs = [torch.tensor(c, dtype=dtype, device="cuda") for c in b]
    y = tt_apply_ad(ws, xs)
    r2 = tt_inner_ad(y, y) - 2 * tt_inner_ad(y, bs) + tt_inner_ad(bs, bs)
    r2.backward()
    ref = grad.residual_loss_grad(structured.laplacian_mpo(2, bits), x, b)
    yw = core.apply_mpo(w, x)
    want = core.inner(yw, yw) - 2 * core.inner(yw, b) + core.inner(b, b)
    # r2 is a difference of three inner products; in FP32 each carries the rounding of
    # y's entries (relative ~1e-7), so the bound scales with the terms, not with r2
    scale = core.inner(yw, yw) + 2 * abs(core.inner(yw, b)) + core.inner(b, b)
    rtol = 1e-12 if dtype == torch.float64 else 1e-6
    assert abs(float(r2) - want) <= rtol * scale
    assert _close([p.grad for p in xs], ref, tol)


def test_hadamard_gradient_through_inner(cuda_lib):
    x = inputs.random_tt(220, 7, 2, 3)
    y = inputs.random_tt(221, 7, 2, 2)
    p = inputs.random_tt(222, 7, 2, 4)
    xs, ys = _params(x), _params(y)
    ps = [torch.tensor(c, device="cuda") for c in p]
    v = tt_inner_ad(tt_hadamard_ad(xs, ys), ps)
    v.backward()
    z = core.hadamard(x, y)
    dz, _ = grad.inner_vjp(z, p, 1.0)
    rx, ry = grad.hadamard_vjp(x, y, dz)
    assert _close([q.grad for q in xs], rx, 1e-10)
    assert _close([q.grad for q in ys], ry, 1e-10)


def test_eval_full_size_sampled(cuda_lib):
    """2^20 samples, L = 40 (2 x 20 bits interleaved), rank 64, FP32 cores."""
    tt = cuda_lib
    L, n = 40, 1 << 20
    x = [c.astype(np.float32) for c in inputs.random_tt(230, L, 2, 64)]
    dg = inputs.random_digits(231, n, [2] * L)
    v = tt.tt_eval(tt.TT.from_numpy(x, dtype=torch.float32), torch.as_tensor(dg, device="cuda"))
    got = v.cpu().double().numpy()
    idx = np.random.default_rng(232).choice(n, 4096, replace=False)
    ref = core.evaluate([c.astype(np.float64) for c in x], dg[idx])
    rms = np.sqrt(np.mean(ref ** 2))
    assert np.max(np.abs(got[idx] - ref)) <= 1e-5 * rms * 4


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-10), (torch.float32, 1e-4)])
def test_residual_gradient_full_size(cuda_lib, dtype, tol):
    """||A x - b||^2 at the fitting workload's size: L = 40 (2 x 20 bits), rank 64, the 2D
    Laplacian (rank 5, so A x has rank 320), b of rank 16; gradient w.r.t. the cores of x."""
    bits = 20
    L = 2 * bits
    w = qtt.laplacian_mpo(2, bits)
    x = inputs.random_tt(240, L, 2, 64)
    b = inputs.random_tt(241, L, 2, 16)
    if dtype == torch.float32:
        x = [c.astype(np.float32).astype(np.float64) for c in x]
        b = [c.astype(np.float32).astype(np.float64) for c in b]
        w = [c.astype(np.float32).astype(np.float64) for c in w]
    ws = [torch.tensor(c, dtype=dtype, device="cuda") for c in w]
    xs = _params(x, dtype)
    bs = [torch.tensor(c, dtype=dtype, device="cuda") for c in b]
    y = tt_apply_ad(ws, xs)
    r2 = tt_inner_ad(y, y) - 2 * tt_inner_ad(y, bs) + tt_inner_ad(bs, bs)
    r2.backward()
    ref = grad.residual_loss_grad(w, x, b)
    assert _close([p.grad for p in xs], ref, tol)


def test_fit_gradient_full_size(cuda_lib):
    """The fit gradient at 2^20 samples, L = 40, rank 64, FP32: the oracle's gradient on the
    first 8192 samples against the GPU's on the same samples, and the full-batch GPU gradient
    against the sum of its gradients over 128 sample blocks (the gradient is linear in the
    per-sample weights, so the blocks must add up to the whole)."""
    tt = cuda_lib
    bits, n, blk = 20, 1 << 20, 8192
    L = 2 * bits
    x = [c.astype(np.float32) for c in inputs.random_tt(250, L, 2, 64)]
    x64 = [c.astype(np.float64) for c in x]
    dg = inputs.random_digits(251, n, [2] * L)
    f = inputs.fit_targets(dg, bits)
    X = tt.TT.from_numpy(x, dtype=torch.float32)
    d = torch.as_tensor(dg, device="cuda")
    v = tt.tt_eval(X, d)
    w = (v.double() - torch.as_tensor(f, device="cuda")) / n
    g_full = tt.tt_eval_backward(X, d, w.float())
    # parity with the oracle on one block
    g0 = tt.tt_eval_backward(X, d[:blk], w[:blk].float())
    ref0 = grad.evaluate_vjp(x64, dg[:blk], w[:blk].cpu().numpy())
    assert _close(g0.cores, ref0, 1e-4)
    # linearity in the samples over the whole batch
    acc = [np.zeros(c.shape) for c in x]
    for s0 in range(0, n, blk):
        gb = tt.tt_eval_backward(X, d[s0:s0 + blk], w[s0:s0 + blk].float())
        for a, c in zip(acc, gb.cores):
            a += c.double().cpu().numpy()
    assert _close(g_full.cores, acc, 1e-5)
