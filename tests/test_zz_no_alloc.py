"""The inner product entry point that allocates nothing (tt_inner_noalloc).

It is for callers that cannot give the library device memory: the environment
scratch is a fixed array inside the library.  Checked against tt_inner (the entry
point that takes a workspace) on two calls in a row, within the tolerance the inner
parity tests use, and for its clean rejection of trains too large for the array.
Collected last so that a failure here comes after every other test has run.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2602_20226_gb300 import api, inputs

pytestmark = pytest.mark.gpu


def _noalloc(lib, X, Y):
    a, b = api._desc(X), api._desc(Y)
    out = ctypes.c_double(0.0)
    code = lib.tt_inner_noalloc(a.ref(), b.ref(), ctypes.byref(out), api._stream_ptr())
    return code, out.value


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_inner_noalloc_matches_tt_inner_twice(cuda_lib, dtype):
    tt = cuda_lib
    lib = tt.load()
    x = inputs.random_tt(300, 40, 2, 64)
    y = inputs.random_tt(301, 40, 2, 16)
    X = tt.TT.from_numpy(x, dtype=dtype)
    Y = tt.TT.from_numpy(y, dtype=dtype)
    ref = tt.tt_inner(X, Y)
    scale = np.sqrt(abs(tt.tt_inner(X, X)) * abs(tt.tt_inner(Y, Y)))
    for _ in range(2):
        code, v = _noalloc(lib, X, Y)
        assert code == 0, lib.tt_last_error()
        assert abs(v - ref) <= 1e-12 * scale, (v, ref)
    # a different pair right after: the scratch keeps the previous call's contents
    z = tt.TT.from_numpy(inputs.random_tt(302, 12, 2, 7), dtype=dtype)
    code, v = _noalloc(lib, z, z)
    assert code == 0
    assert abs(v - tt.tt_inner(z, z)) <= 1e-12 * abs(v)


def test_inner_noalloc_rejects_oversized(cuda_lib):
    tt = cuda_lib
    lib = tt.load()
    big = tt.TT.from_numpy(inputs.random_tt(303, 3, 2, [1, 600, 600, 1]))
    code, _ = _noalloc(lib, big, big)
    assert code == 4  # TT_ERR_UNSUPPORTED
    assert b"fixed" in lib.tt_last_error()
