"""ctypes view of the C ABI declared in include/tt.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libtt.so")

TT_OK = 0
TT_ERR_ARG, TT_ERR_SHAPE, TT_ERR_DTYPE, TT_ERR_UNSUPPORTED = 1, 2, 3, 4
TT_ERR_WORKSPACE, TT_ERR_CUDA, TT_ERR_NUMERIC, TT_ERR_TIMEOUT = 5, 6, 7, 8
STATUS_NAMES = {
    0: "TT_OK",
    1: "TT_ERR_ARG",
    2: "TT_ERR_SHAPE",
    3: "TT_ERR_DTYPE",
    4: "TT_ERR_UNSUPPORTED",
    5: "TT_ERR_WORKSPACE",
    6: "TT_ERR_CUDA",
    7: "TT_ERR_NUMERIC",
    8: "TT_ERR_TIMEOUT",
}
TT_F64, TT_F32 = 0, 1
TT_PREC_FP64, TT_PREC_MIXED = 0, 1
TT_MAX_SITES = 128
TT_MAX_MODE = 16


class tt_train(ctypes.Structure):
    _fields_ = [
        ("L", ctypes.c_int32),
        ("dtype", ctypes.c_int32),
        ("d", ctypes.POINTER(ctypes.c_int32)),
        ("ranks", ctypes.POINTER(ctypes.c_int64)),
        ("cores", ctypes.POINTER(ctypes.c_void_p)),
    ]


class tt_mpo(ctypes.Structure):
    _fields_ = [
        ("L", ctypes.c_int32),
        ("dtype", ctypes.c_int32),
        ("d", ctypes.POINTER(ctypes.c_int32)),
        ("ranks", ctypes.POINTER(ctypes.c_int64)),
        ("cores", ctypes.POINTER(ctypes.c_void_p)),
    ]


P = ctypes.POINTER
vp = ctypes.c_void_p
i32, i64, f64, sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t

SIGNATURES = {
    "tt_last_error": (ctypes.c_char_p, []),
    "tt_version": (ctypes.c_char_p, []),
    "tt_launch_count": (ctypes.c_uint64, []),
    "tt_profile_enable": (None, [i32]),
    "tt_profile_read": (ctypes.c_int, [i32, P(f64), P(f64), P(ctypes.c_uint64)]),
    "tt_profile_read_executed": (ctypes.c_int, [i32, P(f64)]),
    "tt_debug_wait_expiry": (ctypes.c_int, [i64, vp, vp]),
    "tt_round_backward_workspace_size": (sz, [P(tt_train)]),
    "tt_round_backward": (ctypes.c_int, [P(tt_train), f64, i64, P(tt_train), P(tt_train), vp, sz, vp]),
    "tt_apply_mpo": (ctypes.c_int, [P(tt_mpo), P(tt_train), P(tt_train), vp]),
    "tt_hadamard": (ctypes.c_int, [P(tt_train), P(tt_train), P(tt_train), vp]),
    "tt_round_workspace_size": (sz, [P(tt_train), i32]),
    "tt_round": (ctypes.c_int, [P(tt_train), f64, i64, i32, P(tt_train), P(f64), vp, sz, vp]),
    "tt_inner_workspace_size": (sz, [P(tt_train), P(tt_train)]),
    "tt_inner": (ctypes.c_int, [P(tt_train), P(tt_train), P(f64), vp, sz, vp]),
    "tt_inner_noalloc": (ctypes.c_int, [P(tt_train), P(tt_train), P(f64), vp]),
    "tt_eval": (ctypes.c_int, [P(tt_train), vp, i64, vp, vp]),
    "tt_apply_mpo_backward": (ctypes.c_int, [P(tt_mpo), P(tt_train), P(tt_train), P(tt_mpo), P(tt_train), vp]),
    "tt_hadamard_backward": (ctypes.c_int, [P(tt_train), P(tt_train), P(tt_train), P(tt_train), P(tt_train), vp]),
    "tt_inner_backward": (ctypes.c_int, [P(tt_train), P(tt_train), f64, P(tt_train), P(tt_train), vp, sz, vp]),
    "tt_eval_backward_workspace_size": (sz, [P(tt_train), i64]),
    "tt_eval_backward": (ctypes.c_int, [P(tt_train), vp, i64, vp, P(tt_train), vp, sz, vp]),
    "tt_apply_round_batched_workspace_size": (sz, [i32, P(tt_mpo), P(tt_train), i32, i32]),
    "tt_apply_round_batched": (ctypes.c_int, [i32, P(tt_mpo), P(tt_train), P(tt_train), f64, i64, i32,
                                              P(tt_train), vp, sz, P(vp), i32]),
    "tt_gemm_f32": (ctypes.c_int, [i32, i32, i32, f64, vp, i64, i64, vp, i64, i64, f64, vp, i64, i64, vp]),
    "tt_gemm_f32_sliced": (ctypes.c_int, [i32, i32, i32, f64, vp, i64, i64, vp, i64, i64, f64, vp, i64, i64, vp]),
}

_lib = None


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libtt.so; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(
            f"libtt.so not found at {p}; build it with `python -m paper_2602_20226_gb300.build`")
    import torch  # noqa: F401  (loads the CUDA runtime torch links against first)

    lib = ctypes.CDLL(p, mode=ctypes.RTLD_GLOBAL)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols() -> list[str]:
    return list(SIGNATURES)
