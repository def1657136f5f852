"""GB300-native quantics tensor-train arithmetic (trainsum's data-parallel hot path).

The compute lives in libtt.so (hand-written sm_103a CUDA behind a C ABI, see
include/tt.h).  This package is the thin Python binding with the same names, plus
the host-side constructors of structured operators and the seeded inputs.
"""
from ._abi import TT_F32, TT_F64, TT_PREC_FP64, TT_PREC_MIXED  # noqa: F401
from .api import (  # noqa: F401
    MPO,
    TT,
    TTError,
    gemm_f32,
    load,
    tt_apply_mpo,
    tt_apply_mpo_backward,
    tt_apply_round_batched,
    tt_eval,
    tt_eval_backward,
    tt_hadamard,
    tt_hadamard_backward,
    tt_inner,
    tt_inner_backward,
    tt_round,
    tt_round_backward,
    tt_round_workspace_size,
)
