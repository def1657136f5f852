"""torch.autograd.Function wrappers over the library's hand-written adjoints.

Each Function's forward and backward are single calls into libtt (tt_eval /
tt_eval_backward, tt_inner / tt_inner_backward, tt_apply_mpo / tt_apply_mpo_backward,
tt_hadamard / tt_hadamard_backward); torch only carries the cores and the graph.
Cores are passed as separate tensors so that each receives its own gradient.

    loss = ((tt_eval_ad(cores, digits) - f) ** 2).mean() / 2      # TT fitting
    y = tt_apply_ad(w_cores, x_cores)                              # A x
    r2 = tt_inner_ad(y, y) - 2 * tt_inner_ad(y, b) + tt_inner_ad(b, b)   # ||A x - b||^2
"""
from __future__ import annotations

import torch

from . import api


def _tt(cores) -> api.TT:
    return api.TT([c.detach().contiguous() for c in cores])


class _Eval(torch.autograd.Function):
    @staticmethod
    def forward(ctx, digits, *cores):
        x = _tt(cores)
        ctx.save_for_backward(digits, *x.cores)
        return api.tt_eval(x, digits)

    @staticmethod
    def backward(ctx, dvalues):
        digits, *cores = ctx.saved_tensors
        g = api.tt_eval_backward(api.TT(list(cores)), digits, dvalues.contiguous())
        return (None, *g.cores)


class _Inner(torch.autograd.Function):
    @staticmethod
    def forward(ctx, nx, *cores):
        x, y = _tt(cores[:nx]), _tt(cores[nx:])
        ctx.nx = nx
        ctx.save_for_backward(*x.cores, *y.cores)
        v = api.tt_inner(x, y)
        return torch.tensor(v, dtype=torch.float64, device=x.device)

    @staticmethod
    def backward(ctx, dout):
        saved = ctx.saved_tensors
        x, y = api.TT(list(saved[:ctx.nx])), api.TT(list(saved[ctx.nx:]))
        want_x = any(ctx.needs_input_grad[1:1 + ctx.nx])
        want_y = any(ctx.needs_input_grad[1 + ctx.nx:])
        gx, gy = api.tt_inner_backward(x, y, float(dout), want_x=want_x, want_y=want_y)
        gxs = gx.cores if gx is not None else [None] * x.L
        gys = gy.cores if gy is not None else [None] * y.L
        return (None, *gxs, *gys)


class _Apply(torch.autograd.Function):
    @staticmethod
    def forward(ctx, nw, *cores):
        W = api.MPO([c.detach().contiguous() for c in cores[:nw]])
        x = _tt(cores[nw:])
        ctx.nw = nw
        ctx.save_for_backward(*W.cores, *x.cores)
        y = api.tt_apply_mpo(W, x).cores
        ctx.yshapes = [c.shape for c in y]
        return tuple(y)

    @staticmethod
    def backward(ctx, *dy):
        saved = ctx.saved_tensors
        W, x = api.MPO(list(saved[:ctx.nw])), api.TT(list(saved[ctx.nw:]))
        want_w = any(ctx.needs_input_grad[1:1 + ctx.nw])
        dyt = api.TT([(d if d is not None else torch.zeros(sh, dtype=x.dtype, device=x.device)).contiguous()
                      for d, sh in zip(dy, ctx.yshapes)])
        gx, gw = api.tt_apply_mpo_backward(W, x, dyt, want_w=want_w)
        gws = gw.cores if gw is not None else [None] * W.L
        return (None, *gws, *gx.cores)


class _Hadamard(torch.autograd.Function):
    @staticmethod
    def forward(ctx, nx, *cores):
        x, y = _tt(cores[:nx]), _tt(cores[nx:])
        ctx.nx = nx
        ctx.save_for_backward(*x.cores, *y.cores)
        z = api.tt_hadamard(x, y).cores
        ctx.zshapes = [c.shape for c in z]
        return tuple(z)

    @staticmethod
    def backward(ctx, *dz):
        saved = ctx.saved_tensors
        x, y = api.TT(list(saved[:ctx.nx])), api.TT(list(saved[ctx.nx:]))
        dzt = api.TT([(d if d is not None else torch.zeros(sh, dtype=x.dtype, device=x.device)).contiguous()
                      for d, sh in zip(dz, ctx.zshapes)])
        gx, gy = api.tt_hadamard_backward(x, y, dzt)
        return (None, *gx.cores, *gy.cores)


def tt_eval_ad(cores, digits):
    """Values of the TT at digit tuples, differentiable w.r.t. the cores."""
    return _Eval.apply(digits, *cores)


def tt_inner_ad(x_cores, y_cores):
    """<x, y> as a 0-d FP64 tensor, differentiable w.r.t. both sets of cores."""
    return _Inner.apply(len(x_cores), *x_cores, *y_cores)


def tt_apply_ad(w_cores, x_cores):
    """Cores of W x, differentiable w.r.t. the operator and the TT cores."""
    return list(_Apply.apply(len(w_cores), *w_cores, *x_cores))


def tt_hadamard_ad(x_cores, y_cores):
    """Cores of x (.) y, differentiable w.r.t. both."""
    return list(_Hadamard.apply(len(x_cores), *x_cores, *y_cores))
