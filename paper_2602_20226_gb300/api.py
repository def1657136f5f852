"""Python binding of libtt with the C-ABI names.

Argument marshalling only: every arithmetic step runs inside libtt's CUDA
kernels.  PyTorch provides the device memory (cores, outputs, workspaces) and the
stream (the current torch stream).  If the library is missing the calls raise;
there is no CPU path.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _abi

_DT = {torch.float64: _abi.TT_F64, torch.float32: _abi.TT_F32}


class TTError(RuntimeError):
    def __init__(self, fn: str, code: int, msg: str):
        super().__init__(f"{fn} -> {_abi.STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def _check(fn: str, code: int) -> None:
    if code != _abi.TT_OK:
        msg = _abi.load().tt_last_error().decode(errors="replace")
        raise TTError(fn, code, msg)


def _stream_ptr(stream=None) -> ctypes.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


@dataclass
class TT:
    """A tensor train whose cores G_k (r_{k-1}, d_k, r_k) are contiguous CUDA tensors."""

    cores: list

    @property
    def L(self) -> int:
        return len(self.cores)

    @property
    def dims(self) -> list[int]:
        return [int(c.shape[1]) for c in self.cores]

    @property
    def ranks(self) -> list[int]:
        return [int(self.cores[0].shape[0])] + [int(c.shape[2]) for c in self.cores]

    @property
    def dtype(self):
        return self.cores[0].dtype

    @property
    def device(self):
        return self.cores[0].device

    @staticmethod
    def from_numpy(cores, device="cuda", dtype=torch.float64) -> "TT":
        return TT([torch.as_tensor(np.ascontiguousarray(c), dtype=dtype, device=device) for c in cores])

    def numpy(self) -> list[np.ndarray]:
        return [c.detach().to("cpu", torch.float64).numpy() for c in self.cores]

    def zeros_like(self) -> "TT":
        return TT([torch.zeros_like(c) for c in self.cores])

    def numel(self) -> int:
        return sum(c.numel() for c in self.cores)


@dataclass
class MPO:
    """A matrix product operator with cores W_k (a_{k-1}, d_k, d_k, a_k) on the device."""

    cores: list

    @property
    def L(self) -> int:
        return len(self.cores)

    @property
    def dims(self) -> list[int]:
        return [int(c.shape[1]) for c in self.cores]

    @property
    def ranks(self) -> list[int]:
        return [int(self.cores[0].shape[0])] + [int(c.shape[3]) for c in self.cores]

    @property
    def dtype(self):
        return self.cores[0].dtype

    @staticmethod
    def from_numpy(cores, device="cuda", dtype=torch.float64) -> "MPO":
        return MPO([torch.as_tensor(np.ascontiguousarray(c), dtype=dtype, device=device) for c in cores])

    def numpy(self) -> list[np.ndarray]:
        return [c.detach().to("cpu", torch.float64).numpy() for c in self.cores]


class _Desc:
    """Keeps the ctypes arrays of one descriptor alive."""

    def __init__(self, cores, dims, ranks, dtype, is_mpo=False):
        L = len(dims)
        self.d = (ctypes.c_int32 * L)(*dims)
        self.r = (ctypes.c_int64 * (L + 1))(*ranks)
        self.p = (ctypes.c_void_p * L)(*[int(c.data_ptr()) if c is not None else 0 for c in cores])
        cls = _abi.tt_mpo if is_mpo else _abi.tt_train
        self.s = cls(L, _DT[dtype], self.d, self.r, self.p)

    def ref(self):
        return ctypes.byref(self.s)

    def ranks(self) -> list[int]:
        return [int(v) for v in self.r]


def _desc(t) -> _Desc:
    for c in t.cores:
        if not c.is_cuda or not c.is_contiguous():
            raise ValueError("cores must be contiguous CUDA tensors")
    return _Desc(t.cores, t.dims, t.ranks, t.dtype, is_mpo=isinstance(t, MPO))


def load():
    return _abi.load()


# ---------------------------------------------------------------------------- forward


def tt_apply_mpo(W: MPO, x: TT, stream=None) -> TT:
    """y = W x, Y_k[(a,r), i, (a',r')] = sum_j W_k[a,i,j,a'] G_k[r,j,r'] (one launch)."""
    lib = load()
    ranks = [a * r for a, r in zip(W.ranks, x.ranks)]
    y = TT([torch.empty((ranks[k], x.dims[k], ranks[k + 1]), dtype=x.dtype, device=x.device)
            for k in range(x.L)])
    dw, dx, dy = _desc(W), _desc(x), _desc(y)
    _check("tt_apply_mpo", lib.tt_apply_mpo(dw.ref(), dx.ref(), dy.ref(), _stream_ptr(stream)))
    return y


def tt_hadamard(x: TT, y: TT, stream=None) -> TT:
    """z = x (.) y, Z_k[(r,s), i, (r',s')] = X_k[r,i,r'] Y_k[s,i,s'] (one launch)."""
    lib = load()
    ranks = [a * b for a, b in zip(x.ranks, y.ranks)]
    z = TT([torch.empty((ranks[k], x.dims[k], ranks[k + 1]), dtype=x.dtype, device=x.device)
            for k in range(x.L)])
    dx, dy, dz = _desc(x), _desc(y), _desc(z)
    _check("tt_hadamard", lib.tt_hadamard(dx.ref(), dy.ref(), dz.ref(), _stream_ptr(stream)))
    return z


def tt_round_workspace_size(x: TT, prec: int) -> int:
    return int(load().tt_round_workspace_size(_desc(x).ref(), prec))


def tt_round(x: TT, eps: float, max_rank: int = 0, prec: int | None = None, stream=None,
             workspace: torch.Tensor | None = None, out_buffers: list | None = None):
    """Rounded copy of x: returns (TT, ||x||).  prec defaults to FP64 for float64
    cores and to the mixed form for float32 cores."""
    lib = load()
    if prec is None:
        prec = _abi.TT_PREC_FP64 if x.dtype == torch.float64 else _abi.TT_PREC_MIXED
    dx = _desc(x)
    need = int(lib.tt_round_workspace_size(dx.ref(), prec))
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=x.device)
    if out_buffers is None:
        out_buffers = [torch.empty(c.numel(), dtype=x.dtype, device=x.device) for c in x.cores]
    od = _Desc(out_buffers, x.dims, x.ranks, x.dtype)
    nrm = ctypes.c_double(0.0)
    code = lib.tt_round(dx.ref(), float(eps), int(max_rank), int(prec), od.ref(), ctypes.byref(nrm),
                        ctypes.c_void_p(workspace.data_ptr()), ctypes.c_size_t(workspace.numel()),
                        _stream_ptr(stream))
    _check("tt_round", code)
    r = od.ranks()
    cores = [out_buffers[k][: r[k] * x.dims[k] * r[k + 1]].view(r[k], x.dims[k], r[k + 1])
             for k in range(x.L)]
    return TT(cores), float(nrm.value)


def tt_inner(x: TT, y: TT, stream=None, workspace: torch.Tensor | None = None) -> float:
    """<x, y> with FP64 environments."""
    lib = load()
    dx, dy = _desc(x), _desc(y)
    need = int(lib.tt_inner_workspace_size(dx.ref(), dy.ref()))
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=x.device)
    out = ctypes.c_double(0.0)
    _check("tt_inner", lib.tt_inner(dx.ref(), dy.ref(), ctypes.byref(out),
                                    ctypes.c_void_p(workspace.data_ptr()),
                                    ctypes.c_size_t(workspace.numel()), _stream_ptr(stream)))
    return float(out.value)


def tt_eval(x: TT, digits: torch.Tensor, stream=None, out: torch.Tensor | None = None) -> torch.Tensor:
    """Entries of x at the index tuples digits (uint8 [n, L], device)."""
    lib = load()
    if digits.dtype != torch.uint8 or not digits.is_cuda or not digits.is_contiguous():
        raise ValueError("digits must be a contiguous uint8 CUDA tensor [n, L]")
    n = int(digits.shape[0])
    if out is None:
        out = torch.empty(n, dtype=x.dtype, device=x.device)
    dx = _desc(x)
    _check("tt_eval", lib.tt_eval(dx.ref(), ctypes.c_void_p(digits.data_ptr()), n,
                                  ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
    return out


def gemm_f32(A: torch.Tensor, B: torch.Tensor, C: torch.Tensor | None = None, alpha: float = 1.0,
             beta: float = 0.0, form: str = "sliced", stream=None) -> torch.Tensor:
    """C = alpha A B + beta C for 2-D FP32 CUDA tensors (any strides) on the tensor cores:
    form "sliced" (tt_gemm_f32_sliced, exact tensor-core sums) or "tf32x3" (tt_gemm_f32)."""
    lib = load()
    fn = {"sliced": "tt_gemm_f32_sliced", "tf32x3": "tt_gemm_f32"}[form]
    M, K = A.shape
    N = B.shape[1]
    if B.shape[0] != K or any(t.dtype != torch.float32 or not t.is_cuda for t in (A, B)):
        raise ValueError("gemm_f32: A (M, K) and B (K, N) must be FP32 CUDA tensors")
    if C is None:
        if beta != 0.0:
            raise ValueError("gemm_f32: beta != 0 needs C")
        C = torch.empty(M, N, dtype=torch.float32, device=A.device)
    _check(fn, getattr(lib, fn)(M, N, K, alpha, ctypes.c_void_p(A.data_ptr()), A.stride(0), A.stride(1),
                                ctypes.c_void_p(B.data_ptr()), B.stride(0), B.stride(1), beta,
                                ctypes.c_void_p(C.data_ptr()), C.stride(0), C.stride(1), _stream_ptr(stream)))
    return C


# ---------------------------------------------------------------------------- adjoints


def tt_apply_mpo_backward(W: MPO, x: TT, dy: TT, want_w: bool = True, stream=None):
    """(dx, dW) of y = W x given dy (fresh zero-initialised gradients)."""
    lib = load()
    gx = x.zeros_like()
    gw = MPO([torch.zeros_like(c) for c in W.cores]) if want_w else None
    dW, dX, dDY, dGX = _desc(W), _desc(x), _desc(dy), _desc(gx)
    dGW = _desc(gw) if want_w else None
    _check("tt_apply_mpo_backward",
           lib.tt_apply_mpo_backward(dW.ref(), dX.ref(), dDY.ref(), dGW.ref() if dGW else None,
                                     dGX.ref(), _stream_ptr(stream)))
    return gx, gw


def tt_hadamard_backward(x: TT, y: TT, dz: TT, stream=None):
    lib = load()
    gx, gy = x.zeros_like(), y.zeros_like()
    a, b, c, d, e = _desc(x), _desc(y), _desc(dz), _desc(gx), _desc(gy)
    _check("tt_hadamard_backward",
           lib.tt_hadamard_backward(a.ref(), b.ref(), c.ref(), d.ref(), e.ref(), _stream_ptr(stream)))
    return gx, gy


def tt_inner_backward(x: TT, y: TT, dout: float = 1.0, want_x=True, want_y=True, stream=None):
    lib = load()
    gx = x.zeros_like() if want_x else None
    gy = y.zeros_like() if want_y else None
    a, b = _desc(x), _desc(y)
    c = _desc(gx) if want_x else None
    d = _desc(gy) if want_y else None
    need = int(lib.tt_inner_workspace_size(a.ref(), b.ref()))
    ws = torch.empty(need, dtype=torch.uint8, device=x.device)
    _check("tt_inner_backward",
           lib.tt_inner_backward(a.ref(), b.ref(), float(dout), c.ref() if c else None,
                                 d.ref() if d else None, ctypes.c_void_p(ws.data_ptr()),
                                 ctypes.c_size_t(need), _stream_ptr(stream)))
    return gx, gy


def tt_round_backward(x: TT, eps: float, dout: TT, max_rank: int = 0, stream=None) -> TT:
    """Gradient w.r.t. the cores of x of a loss of tt_round(x, eps, max_rank) (FP64 form),
    given its gradient dout w.r.t. the rounded cores (fresh zero-initialised result)."""
    lib = load()
    gx = x.zeros_like()
    a, b, c = _desc(x), _desc(dout), _desc(gx)
    need = int(lib.tt_round_backward_workspace_size(a.ref()))
    ws = torch.empty(max(need, 1), dtype=torch.uint8, device=x.device)
    _check("tt_round_backward",
           lib.tt_round_backward(a.ref(), float(eps), int(max_rank), b.ref(), c.ref(),
                                 ctypes.c_void_p(ws.data_ptr()), ctypes.c_size_t(need), _stream_ptr(stream)))
    return gx


def tt_eval_backward(x: TT, digits: torch.Tensor, dvalues: torch.Tensor, stream=None) -> TT:
    lib = load()
    n = int(digits.shape[0])
    gx = x.zeros_like()
    a, b = _desc(x), _desc(gx)
    need = int(lib.tt_eval_backward_workspace_size(a.ref(), n))
    ws = torch.empty(max(need, 1), dtype=torch.uint8, device=x.device)
    dv = dvalues.to(x.dtype).contiguous()
    _check("tt_eval_backward",
           lib.tt_eval_backward(a.ref(), ctypes.c_void_p(digits.data_ptr()), n,
                                ctypes.c_void_p(dv.data_ptr()), b.ref(), ctypes.c_void_p(ws.data_ptr()),
                                ctypes.c_size_t(need), _stream_ptr(stream)))
    return gx


# ---------------------------------------------------------------------------- batched


def tt_apply_round_batched(Ws: list, xs: list, eps: float, max_rank: int = 0, prec: int | None = None,
                           nstreams: int = 5, workspace: torch.Tensor | None = None,
                           streams: list | None = None):
    """Apply each W[i] to x[i] and round, for many trains at once (tt_apply_round_batched).

    Returns the list of rounded TTs.  The trains advance in lock-step inside the library on
    the first stream; up to four more streams run the size classes of the bond SVDs side by
    side.  Every buffer comes from torch.
    """
    lib = load()
    n = len(xs)
    if n == 0:
        return []
    dtype, dev = xs[0].dtype, xs[0].device
    if prec is None:
        prec = _abi.TT_PREC_FP64 if dtype == torch.float64 else _abi.TT_PREC_MIXED
    wd = [_desc(W) for W in Ws]
    xd = [_desc(x) for x in xs]
    # the apply outputs and the rounded results of all trains are carved from two flat
    # buffers (two allocations per call instead of two per core); each core starts on a
    # 256-byte boundary
    rks = [[a * b for a, b in zip(W.ranks, x.ranks)] for W, x in zip(Ws, xs)]
    quantum = 256 // torch.empty((), dtype=dtype).element_size()
    sizes = [[-(-(r[k] * x.dims[k] * r[k + 1]) // quantum) * quantum for k in range(x.L)] for r, x in zip(rks, xs)]
    total = sum(sum(z) for z in sizes)
    yflat = torch.empty(max(total, 1), dtype=dtype, device=dev)
    oflat = torch.empty(max(total, 1), dtype=dtype, device=dev)
    ys, yd, ob, od = [], [], [], []
    off = 0
    for x, r, z in zip(xs, rks, sizes):
        y, bufs = [], []
        for k in range(x.L):
            m = r[k] * x.dims[k] * r[k + 1]
            y.append(yflat[off: off + m].view(r[k], x.dims[k], r[k + 1]))
            bufs.append(oflat[off: off + m])
            off += z[k]
        ys.append(y)
        yd.append(_Desc(y, x.dims, r, dtype))
        ob.append(bufs)
        od.append(_Desc(bufs, x.dims, r, dtype))
    Warr = (_abi.tt_mpo * n)(*[d.s for d in wd])
    Xarr = (_abi.tt_train * n)(*[d.s for d in xd])
    Yarr = (_abi.tt_train * n)(*[d.s for d in yd])
    Oarr = (_abi.tt_train * n)(*[d.s for d in od])
    need = int(lib.tt_apply_round_batched_workspace_size(n, Warr, Xarr, int(prec), int(nstreams)))
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
    if streams is None:
        streams = [torch.cuda.Stream(device=dev) for _ in range(nstreams)]
    sarr = (ctypes.c_void_p * nstreams)(*[s.cuda_stream for s in streams])
    torch.cuda.current_stream(dev).synchronize()
    code = lib.tt_apply_round_batched(n, Warr, Xarr, Yarr, float(eps), int(max_rank), int(prec), Oarr,
                                      ctypes.c_void_p(workspace.data_ptr()), ctypes.c_size_t(workspace.numel()),
                                      sarr, int(nstreams))
    _check("tt_apply_round_batched", code)
    outs = []
    for i, x in enumerate(xs):
        r = [int(v) for v in Oarr[i].ranks[: x.L + 1]]
        outs.append(TT([ob[i][k][: r[k] * x.dims[k] * r[k + 1]].view(r[k], x.dims[k], r[k + 1])
                        for k in range(x.L)]))
    return outs
