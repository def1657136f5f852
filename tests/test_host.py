"""Host-side checks that need no GPU: the C ABI library loads and exports every
declared entry point, the host constructors agree with the oracle's, and the
seeded inputs are deterministic."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import core, structured
from paper_2602_20226_gb300 import _abi, inputs, qtt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    txt = open(os.path.join(ROOT, "include", "tt.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(tt_[a-z_0-9]+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _header_functions()
    for want in ["tt_apply_mpo", "tt_hadamard", "tt_round", "tt_inner", "tt_eval",
                 "tt_apply_mpo_backward", "tt_hadamard_backward", "tt_inner_backward",
                 "tt_eval_backward", "tt_last_error"]:
        assert want in names


def test_library_exports_every_declared_symbol():
    if not os.path.exists(_abi.LIB_PATH):
        from paper_2602_20226_gb300 import build

        build.build()
    lib = ctypes.CDLL(_abi.LIB_PATH)
    for name in _header_functions():
        assert hasattr(lib, name), name
    # the binding declares a signature for every header function
    assert set(_header_functions()) <= set(_abi.exported_symbols())


def test_library_validates_on_host_without_gpu():
    """Argument validation runs before any CUDA call, so it works on a CPU-only host."""
    lib = _abi.load()
    assert lib.tt_apply_mpo(None, None, None, None) == 1  # TT_ERR_ARG
    assert b"NULL" in lib.tt_last_error()
    L = 3
    d = (ctypes.c_int32 * L)(2, 2, 2)
    r = (ctypes.c_int64 * (L + 1))(1, 4, 4, 2)  # bad boundary rank
    p = (ctypes.c_void_p * L)(1, 2, 3)
    x = _abi.tt_train(L, _abi.TT_F64, d, r, p)
    assert lib.tt_eval(ctypes.byref(x), None, 0, None, None) == 2  # TT_ERR_SHAPE
    r2 = (ctypes.c_int64 * (L + 1))(1, 4, 4, 1)
    x2 = _abi.tt_train(L, 7, d, r2, p)
    assert lib.tt_eval(ctypes.byref(x2), None, 0, None, None) == 3  # TT_ERR_DTYPE
    x3 = _abi.tt_train(200, _abi.TT_F64, d, r2, p)
    assert lib.tt_eval(ctypes.byref(x3), None, 0, None, None) == 4  # TT_ERR_UNSUPPORTED
    x4 = _abi.tt_train(L, _abi.TT_F32, d, r2, p)
    out = _abi.tt_train(L, _abi.TT_F32, d, (ctypes.c_int64 * (L + 1))(1, 4, 4, 1), p)
    # FP64 form on FP32 cores is a dtype error, caught before any launch
    assert lib.tt_round(ctypes.byref(x4), 1e-6, 0, _abi.TT_PREC_FP64, ctypes.byref(out), None,
                        ctypes.c_void_p(1), 1 << 20, None) == 3
    assert lib.tt_round(ctypes.byref(x4), -1.0, 0, _abi.TT_PREC_MIXED, ctypes.byref(out), None,
                        ctypes.c_void_p(1), 1 << 20, None) == 1
    assert lib.tt_round_workspace_size(ctypes.byref(x2), 0) == 0


def test_gemm_and_batched_entries_validate_on_host_without_gpu():
    lib = _abi.load()
    vp = ctypes.c_void_p
    for fn in ("tt_gemm_f32_sliced", "tt_gemm_f32"):
        f = getattr(lib, fn)
        # negative size
        assert f(-1, 4, 4, 1.0, vp(1), 4, 1, vp(1), 4, 1, 0.0, vp(1), 4, 1, None) == 1
        # NULL operand with K > 0
        assert f(4, 4, 4, 1.0, None, 4, 1, vp(1), 4, 1, 0.0, vp(1), 4, 1, None) == 1
        assert b"NULL" in lib.tt_last_error()
        # empty output: nothing to do, no device touched
        assert f(0, 4, 4, 1.0, None, 4, 1, None, 4, 1, 0.0, None, 4, 1, None) == 0
    L = 3
    d = (ctypes.c_int32 * L)(2, 2, 2)
    r = (ctypes.c_int64 * (L + 1))(1, 2, 2, 1)
    p = (ctypes.c_void_p * L)(1, 2, 3)
    a = (ctypes.c_int64 * (L + 1))(1, 3, 3, 1)
    W = (_abi.tt_mpo * 1)(_abi.tt_mpo(L, _abi.TT_F32, d, a, p))
    X = (_abi.tt_train * 1)(_abi.tt_train(L, _abi.TT_F32, d, r, p))
    Y = (_abi.tt_train * 1)(_abi.tt_train(L, _abi.TT_F32, d, (ctypes.c_int64 * (L + 1))(1, 6, 6, 1), p))
    O = (_abi.tt_train * 1)(_abi.tt_train(L, _abi.TT_F32, d, (ctypes.c_int64 * (L + 1))(1, 6, 6, 1), p))
    streams = (ctypes.c_void_p * 1)(None)
    f = lib.tt_apply_round_batched
    assert f(-1, W, X, Y, 1e-6, 0, _abi.TT_PREC_MIXED, O, vp(1), 1 << 20, streams, 1) == 1
    assert f(0, None, None, None, 1e-6, 0, _abi.TT_PREC_MIXED, None, None, 0, None, 0) == 0
    assert f(1, W, X, Y, -1.0, 0, _abi.TT_PREC_MIXED, O, vp(1), 1 << 20, streams, 1) == 1  # eps < 0
    assert f(1, W, X, Y, 1e-6, 0, 5, O, vp(1), 1 << 20, streams, 1) == 1  # unknown prec
    assert f(1, W, X, Y, 1e-6, 0, _abi.TT_PREC_FP64, O, vp(1), 1 << 20, streams, 1) == 3  # FP32 cores, FP64 form
    assert f(1, W, X, Y, 1e-6, 0, _abi.TT_PREC_MIXED, O, None, 1 << 20, streams, 1) != 0  # no workspace


@pytest.mark.parametrize("n_dims,bits", [(1, 7), (2, 4), (3, 3), (2, 5)])
def test_laplacian_constructor_matches_oracle(n_dims, bits):
    a = qtt.laplacian_mpo(n_dims, bits)
    b = structured.laplacian_mpo(n_dims, bits)
    assert core.ranks(a) == core.ranks(b)
    assert np.array_equal(core.full_mpo(a), core.full_mpo(b))


@pytest.mark.parametrize("fn", ["exp", "cos", "sin"])
def test_closed_form_constructors_match_oracle(fn):
    bits = 9
    if fn == "exp":
        a = qtt.exp_tt(bits, -1.0, 2.0, 0.7, 0.3)
        b = structured.exp_tt([2] * bits, -1.0, 2.0, 0.7, 0.3)
    elif fn == "cos":
        a = qtt.cos_tt(bits, -1.0, 1.0, 5.0, 0.2)
        b = structured.cos_tt([2] * bits, -1.0, 1.0, 5.0, 0.2)
    else:
        a = qtt.sin_tt(bits, 0.0, 1.0, 2 * np.pi)
        b = structured.sin_tt([2] * bits, 0.0, 1.0, 2 * np.pi)
    assert np.allclose(core.full(a), core.full(b), rtol=1e-14, atol=1e-14)


def test_inputs_are_deterministic():
    a = inputs.random_tt(5, 6, 2, 4)
    b = inputs.random_tt(5, 6, 2, 4)
    assert all(np.array_equal(u, v) for u, v in zip(a, b))
    assert [c.shape for c in a] == [(1, 2, 4)] + [(4, 2, 4)] * 4 + [(4, 2, 1)]
    s = inputs.batch_shapes(1, 64)
    assert all(20 <= L <= 60 and 8 <= r <= 128 and a in (3, 4, 5) for L, r, a in s)
    dg = inputs.random_digits(3, 1000, [2, 3, 5])
    assert dg.dtype == np.uint8 and dg[:, 2].max() == 4 and dg[:, 1].max() == 2


def test_random_tt_norm_is_one_in_expectation():
    norms = [core.norm(inputs.random_tt(s, 8, 2, 4)) ** 2 for s in range(200)]
    assert 0.8 < np.mean(norms) < 1.25


def test_workspace_queries_on_host_without_gpu():
    """The workspace queries are host arithmetic: they answer without a GPU, grow with the
    ranks, hold at least the largest core, and the evaluation adjoint's stops growing at one
    chunk of at most 1 GiB of prefix and suffix states."""
    lib = _abi.load()
    L = 40
    keep = []

    def train(dtype, r):
        d = (ctypes.c_int32 * L)(*([2] * L))
        rk = (ctypes.c_int64 * (L + 1))(*([1] + [r] * (L - 1) + [1]))
        p = (ctypes.c_void_p * L)(*([1] * L))
        keep.append((d, rk, p))
        return ctypes.byref(_abi.tt_train(L, dtype, d, rk, p))

    prev = None
    for r in (8, 64, 320):
        x64, x32 = train(_abi.TT_F64, r), train(_abi.TT_F32, r)
        sizes = (lib.tt_round_workspace_size(x64, _abi.TT_PREC_FP64),
                 lib.tt_round_workspace_size(x32, _abi.TT_PREC_MIXED),
                 lib.tt_round_backward_workspace_size(x64),
                 lib.tt_inner_workspace_size(x64, x64))
        assert sizes[0] >= 8 * r * 2 * r and sizes[1] >= 4 * r * 2 * r
        if prev is not None:
            assert all(a > b for a, b in zip(sizes, prev)), (r, sizes, prev)
        prev = sizes
    x = train(_abi.TT_F32, 64)
    per_sample = (1 + 64 * (L - 1)) + (64 * (L - 1) + 1)  # sum_k r_k + r_{k+1}
    cores = 2 * (2 * 64 + (L - 2) * 64 * 64)
    ns = [1, 1000, 65536, 10 ** 6, 10 ** 8, 2 * 10 ** 8]
    ws = [lib.tt_eval_backward_workspace_size(x, n) for n in ns]
    assert all(b >= a for a, b in zip(ws, ws[1:]))
    assert ws[1] >= 1000 * per_sample * 4
    assert ws[-1] == ws[-2] <= (1 << 30) + 8 * cores + 4096
