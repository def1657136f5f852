"""Failure handling on the GPU, in the forms that fault or hang nothing.

* A bounded device wait on a flag that nothing sets gives up after its poll limit, raises the
  timeout bit of the device status word, and the call returns TT_ERR_TIMEOUT; the context
  stays usable (a rounding right after it is still exact).
* Non-finite input cores (NaN, Inf) come back as TT_ERR_NUMERIC from tt_round and from the
  batched driver, with nothing else disturbed.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import core
from paper_2602_20226_gb300 import _abi, inputs

pytestmark = pytest.mark.gpu


def test_bounded_wait_expires_with_timeout_status(cuda_lib):
    tt = cuda_lib
    lib = tt.load()
    scratch = torch.zeros(4, dtype=torch.int32, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for limit in (1, 1000, 1 << 16):
        code = lib.tt_debug_wait_expiry(limit, ctypes.c_void_p(scratch.data_ptr()), s)
        assert code == _abi.TT_ERR_TIMEOUT, code
        assert b"expired" in lib.tt_last_error()
    assert lib.tt_debug_wait_expiry(0, ctypes.c_void_p(scratch.data_ptr()), s) == _abi.TT_ERR_ARG
    # the context is intact: the next rounding is exact
    x = inputs.random_tt(40, 8, 2, 6)
    Z, _ = tt.tt_round(tt.TT.from_numpy(x), 1e-12)
    assert core.rel_err(Z.numpy(), core.round_tt(x, 1e-12)) <= 1e-12


@pytest.mark.parametrize("bad", [np.nan, np.inf])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_round_non_finite_input(cuda_lib, bad, dtype):
    tt = cuda_lib
    x = inputs.random_tt(41, 9, 2, 5)
    x[4] = x[4].copy()
    x[4][1, 0, 2] = bad
    with pytest.raises(tt.TTError) as ei:
        tt.tt_round(tt.TT.from_numpy(x, dtype=dtype), 1e-8)
    assert ei.value.code == _abi.TT_ERR_NUMERIC
    # a finite train right after it is unaffected
    y = inputs.random_tt(42, 9, 2, 5)
    Z, _ = tt.tt_round(tt.TT.from_numpy(y, dtype=dtype), 1e-8)
    tol = 1e-12 if dtype == torch.float64 else 1e-6
    assert core.rel_err(Z.numpy(), core.round_tt([c.astype(np.float32).astype(np.float64) for c in y]
                                                 if dtype == torch.float32 else y, 1e-8)) <= tol


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_batched_non_finite_input(cuda_lib, dtype):
    tt = cuda_lib
    xs = [inputs.random_tt(43 + i, L, 2, r) for i, (L, r) in enumerate([(6, 4), (8, 5), (1, 1)])]
    ws = [inputs.random_mpo(53 + i, x.__len__(), 2, 3) for i, x in enumerate(xs)]
    xs[1][3] = xs[1][3].copy()
    xs[1][3][0, 1, 0] = np.nan
    X = [tt.TT.from_numpy(x, dtype=dtype) for x in xs]
    W = [tt.MPO.from_numpy(w, dtype=dtype) for w in ws]
    with pytest.raises(tt.TTError) as ei:
        tt.tt_apply_round_batched(W, X, 1e-6)
    assert ei.value.code == _abi.TT_ERR_NUMERIC
    # one-site train with a non-finite core (no bond SVD to notice it): the norm check does
    xs1 = [[np.full((1, 2, 1), np.inf)]]
    with pytest.raises(tt.TTError) as ei:
        tt.tt_apply_round_batched([tt.MPO.from_numpy(inputs.random_mpo(60, 1, 2, 1), dtype=dtype)],
                                  [tt.TT.from_numpy(xs1[0], dtype=dtype)], 1e-6)
    assert ei.value.code == _abi.TT_ERR_NUMERIC
