"""GPU checks of the tensor-core (tcgen05) GEMMs, 3xTF32 and sliced, and of the mixed form of rounding.

GEMM bound: with x = x_hi + x_lo (x_hi = rn_tf32(x), |x_lo| <= 2^-12 |x|), each product
keeps A_hi B_hi + A_hi B_lo + A_lo B_hi; the dropped A_lo B_lo and the TF32 conversion
of the lo parts cost at most 2^-22 |a b|, and FP32 accumulation of K terms at most
K 2^-24 sum |a b|.  So |C - AB| <= (4 + K) 2^-24 (|A| |B|) elementwise.  The tensor
cores do not accumulate with IEEE round-to-nearest, so the relative RMS error grows
like sqrt(K) 2^-24 times a small factor (measured 4.6e-6 at K = 640); the RMS check
allows 4e-7 sqrt(K), far below the ~1e-4 a TF32-only product (lo terms missing) gives.

Mixed rounding: FP32 cores; every Householder panel factored in FP64 and rounded back to
FP32, with tau and T recomputed in FP64 from the rounded reflectors; the block-reflector
products W1 = V^T X and W2 = T^T W1 in FP64 and the update X -= V W2 with exact products and
float-float sums; the core GEMMs in the sliced tensor-core form where its tiles fill the
GPU and compensated FP32 dot products (Dot2) below that; a bond whose stored factor an
FP64 certificate proves full rank skips its SVD, the others get an FP32 Jacobi (FP64 Jacobi
where it hits its sweep cap); sigma, the truncation and the norm are FP64; compared with
the FP64 oracle run on the same FP32 values.  Stated tolerance: e <= 1e-6 with equal ranks
(the 40-site rank-320 train measured 5.3e-7; a CPU emulation of the chain gives 5.1e-7,
against 2.5e-6 with FP32 Householder panels).  For eps below FP32 resolution the mixed
form drops the noise-level singular values and is held to 2e-6 of the unrounded train.
The 3xTF32 GEMM is not on the rounding path: its MMA results are rounded toward zero, a
bias that added up to 1e-5..4e-5 over the 78 sequential QR/GEMM steps of that train.  The
sliced form's tensor-core sums are sums of small integers, exact whatever the rounding.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import core, structured
from paper_2602_20226_gb300 import inputs, qtt

pytestmark = pytest.mark.gpu


def _gemm(lib, A, B, C, alpha=1.0, beta=0.0, a_cm=False, b_cm=False, fn="tt_gemm_f32"):
    M, K = A.shape
    N = B.shape[1]
    Ad = torch.as_tensor(A.T.copy() if a_cm else A, device="cuda")
    Bd = torch.as_tensor(B.T.copy() if b_cm else B, device="cuda")
    Cd = torch.as_tensor(C, device="cuda")
    sam, sak = (1, M) if a_cm else (K, 1)
    sbk, sbn = (1, K) if b_cm else (N, 1)
    code = getattr(lib, fn)(M, N, K, alpha, ctypes.c_void_p(Ad.data_ptr() if K else 0), sam, sak,
                            ctypes.c_void_p(Bd.data_ptr() if K else 0), sbk, sbn, beta,
                            ctypes.c_void_p(Cd.data_ptr()), N, 1, None)
    assert code == 0, lib.tt_last_error()
    torch.cuda.synchronize()
    return Cd.cpu().numpy()


@pytest.mark.parametrize("M,N,K,a_cm,b_cm", [
    (128, 128, 32, False, False),
    (300, 200, 100, True, False),
    (64, 1000, 77, False, True),   # short M: computed as C^T = B^T A^T
    (1000, 40, 640, True, True),
    (7, 5, 3, False, False),       # tiny: SIMT fallback inside the dispatcher is not used here
    (256, 320, 1280, False, False),
])
def test_gemm_f32_tensor_cores(cuda_lib, M, N, K, a_cm, b_cm):
    lib = cuda_lib.load()
    g = np.random.default_rng(M * 7 + N * 3 + K)
    A = g.standard_normal((M, K)).astype(np.float32)
    B = g.standard_normal((K, N)).astype(np.float32)
    C0 = g.standard_normal((M, N)).astype(np.float32)
    got = _gemm(lib, A, B, C0.copy(), 1.5, -0.5, a_cm, b_cm)
    ref = 1.5 * (A.astype(np.float64) @ B.astype(np.float64)) - 0.5 * C0.astype(np.float64)
    bound = (4 + K) * 2.0 ** -24 * (1.5 * np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64)
                                     + 0.5 * np.abs(C0)) + 1e-30
    err = np.abs(got - ref)
    assert np.all(err <= bound), float((err / bound).max())
    rel_rms = np.sqrt(np.mean(err ** 2) / np.mean(ref ** 2))
    assert rel_rms < 4e-7 * np.sqrt(K) + 1e-7, rel_rms


def test_gemm_f32_twice_identical(cuda_lib):
    lib = cuda_lib.load()
    g = np.random.default_rng(5)
    A = g.standard_normal((500, 300)).astype(np.float32)
    B = g.standard_normal((300, 260)).astype(np.float32)
    a = _gemm(lib, A, B, np.zeros((500, 260), np.float32))
    b = _gemm(lib, A, B, np.zeros((500, 260), np.float32))
    assert np.array_equal(a, b)


def _f32(cores):
    return [c.astype(np.float32).astype(np.float64) for c in cores]


def _mixed_round(tt, y32, eps):
    Y = tt.TT.from_numpy(y32, dtype=torch.float32)
    Z, nrm = tt.tt_round(Y, eps, prec=tt.TT_PREC_MIXED)
    return Z.numpy(), nrm


def test_mixed_round_c1(cuda_lib):
    x = _f32(inputs.random_tt(1, 10, 2, 8))
    y = _f32(core.apply_mpo(structured.laplacian_mpo(1, 10), x))
    ref, info = core.round_tt(y, 1e-6, return_info=True)
    got, nrm = _mixed_round(cuda_lib, y, 1e-6)
    assert abs(nrm - info["norm"]) <= 1e-6 * info["norm"]
    assert core.rel_err(got, ref) <= 1e-6
    assert core.rel_err(got, y) <= 1e-6 * 1.01 + 1e-6


def test_mixed_round_c2_shapes(cuda_lib):
    """L = 40, r = 64, 2D Laplacian (n = 320), eps = 1e-6, FP32 cores."""
    tt = cuda_lib
    x = _f32(inputs.random_tt(2, 40, 2, 64))
    W = qtt.laplacian_mpo(2, 20)
    Y = tt.tt_apply_mpo(tt.MPO.from_numpy(W, dtype=torch.float32), tt.TT.from_numpy(x, dtype=torch.float32))
    y = Y.numpy()
    Z, nrm = tt.tt_round(Y, 1e-6, prec=tt.TT_PREC_MIXED)
    ref, info = core.round_tt(y, 1e-6, return_info=True)
    got = Z.numpy()
    e = core.rel_err(got, ref)
    assert e <= 1e-6, e
    assert Z.ranks == core.ranks(ref)
    assert core.rel_err(got, y) <= 1e-6 * 1.01 + 1e-6
    # orthogonality of the left cores, stated for the mixed form (FP32 storage)
    worst = max(core.left_orthogonality_defect(got[k]) for k in range(0, 39, 5))
    assert worst <= 1e-4, worst


@pytest.mark.parametrize("case", ["modes", "wide_left", "hadamard"])
def test_mixed_round_ragged(cuda_lib, case):
    tt = cuda_lib
    if case == "modes":
        x = _f32(inputs.random_tt(3, 6, [2, 3, 5, 2, 3, 2], [1, 6, 7, 9, 5, 4, 1]))
    elif case == "wide_left":
        x = _f32(inputs.random_tt(8, 5, 2, [1, 40, 40, 40, 40, 1]))
    else:
        h = inputs.random_tt(11, 12, 2, 5)
        x = _f32(core.hadamard(h, h))
    ref = core.round_tt(x, 1e-6)
    got, _ = _mixed_round(tt, x, 1e-6)
    assert core.rel_err(got, ref) <= 1e-6


@pytest.mark.parametrize("case", ["laplacian", "hadamard"])
@pytest.mark.parametrize("eps", [1e-8, 1e-10])
def test_mixed_round_below_fp32_resolution(cuda_lib, case, eps):
    """eps below what FP32 factors resolve: the mixed form drops the noise-level singular
    values (< 2^-22 sigma_1 at each bond) and stays within a few 1e-7 of the train."""
    if case == "laplacian":
        x = _f32(inputs.random_tt(5, 20, 2, 32))
        y = _f32(core.apply_mpo(structured.laplacian_mpo(2, 10), x))
    else:
        h = inputs.random_tt(12, 14, 2, 6)
        y = _f32(core.hadamard(h, h))
    got, nrm = _mixed_round(cuda_lib, y, eps)
    assert all(np.isfinite(c).all() for c in got)
    assert core.rel_err(got, y) <= 2e-6
    assert abs(nrm - core.norm(y)) <= 1e-6 * core.norm(y)


def test_mixed_round_noise_level_columns(cuda_lib):
    """A train of the uneven batch (L = 42, r = 41, random MPO of rank 4) whose bond factors
    carry many singular values at FP32 noise level: the FP32 Jacobi must leave pairs of such
    columns alone (they never become orthogonal in FP32) instead of running into its cap."""
    tt = cuda_lib
    x = _f32(inputs.random_tt(4469, 42, 2, 41))
    w = _f32(inputs.random_mpo(4969, 42, 2, 4))
    y = _f32(core.apply_mpo(w, x))
    got, nrm = _mixed_round(tt, y, 1e-6)
    ref = core.round_tt(y, 1e-6)
    assert all(np.isfinite(c).all() for c in got)
    assert core.ranks(got) == core.ranks(ref)
    assert core.rel_err(got, ref) <= 1e-6


# ---------------------------------------------------------------- sliced (exact-sum) form
# Per 32-wide K block: v = 2^(E-9) (h1 + 2^-9 h2 + 2^-18 h3) + d with |d| <= 2^(E-28) and
# 2^(E-1) <= max|v| < 2^E; the dropped h2 h3, h3 h2, h3 h3 products and the remainders d
# cost at most 2^-25 max|a| max|b| per product, i.e. 2^-20 per block of 32, plus the final
# rounding of the result to FP32 (2^-24 |result|).

def _sliced_bound(A, B):
    K = A.shape[1]
    A64, B64 = np.abs(A.astype(np.float64)), np.abs(B.astype(np.float64))
    bound = np.zeros((A.shape[0], B.shape[1]))
    for k0 in range(0, K, 32):
        bound += np.outer(A64[:, k0:k0 + 32].max(axis=1), B64[k0:k0 + 32].max(axis=0))
    return 2.0 ** -20 * bound + 2.0 ** -40 * (A64 @ B64)


@pytest.mark.parametrize("M,N,K,a_cm,b_cm", [
    (128, 64, 32, False, False),   # one tile, one K block
    (256, 128, 16, True, True),    # one partial K block
    (300, 200, 100, True, False),  # ragged tiles and a ragged last K block
    (64, 1000, 77, False, True),   # short M: computed as C^T = B^T A^T
    (1000, 40, 640, True, True),
    (7, 5, 3, False, False),       # K < 32: one partial block
    (256, 320, 1280, False, False),
    (33, 17, 2000, False, True),   # long K, one small tile
])
def test_gemm_f32_sliced(cuda_lib, M, N, K, a_cm, b_cm):
    lib = cuda_lib.load()
    g = np.random.default_rng(M * 11 + N * 5 + K)
    # magnitudes spread over e^-4..e^4 so that rows and columns get different block exponents
    A = (g.standard_normal((M, K)) * np.exp(g.uniform(-4, 4, (M, K)))).astype(np.float32)
    B = (g.standard_normal((K, N)) * np.exp(g.uniform(-4, 4, (1, N)))).astype(np.float32)
    C0 = g.standard_normal((M, N)).astype(np.float32)
    got = _gemm(lib, A, B, C0.copy(), 1.5, -0.5, a_cm, b_cm, fn="tt_gemm_f32_sliced")
    ref = 1.5 * (A.astype(np.float64) @ B.astype(np.float64)) - 0.5 * C0.astype(np.float64)
    bound = 1.5 * _sliced_bound(A, B) + 2.0 ** -24 * np.abs(ref) + 1e-30
    err = np.abs(got - ref)
    assert np.all(err <= bound), float((err / bound).max())
    # far inside the bound in the mean: the rounding of the FP32 result dominates
    assert np.sqrt(np.mean(err ** 2) / np.mean(ref ** 2)) < 2.0 ** -23


def test_gemm_f32_sliced_integers_exact(cuda_lib):
    """Integer operands with every partial sum below 2^24: the exact product, bit for bit."""
    lib = cuda_lib.load()
    g = np.random.default_rng(17)
    A = g.integers(-64, 65, (200, 1000)).astype(np.float32)
    B = g.integers(-64, 65, (1000, 150)).astype(np.float32)
    got = _gemm(lib, A, B, np.zeros((200, 150), np.float32), fn="tt_gemm_f32_sliced")
    ref = A.astype(np.int64) @ B.astype(np.int64)
    assert np.abs(ref).max() < 2 ** 24
    assert np.array_equal(got.astype(np.int64), ref)


def test_gemm_f32_sliced_unbiased_on_positive_data(cuda_lib):
    """Sums of positive products, where a rounding bias would add up over K = 4096."""
    lib = cuda_lib.load()
    g = np.random.default_rng(23)
    A = g.uniform(0, 1, (256, 4096)).astype(np.float32)
    B = g.uniform(0, 1, (4096, 256)).astype(np.float32)
    got = _gemm(lib, A, B, np.zeros((256, 256), np.float32), fn="tt_gemm_f32_sliced")
    ref = A.astype(np.float64) @ B.astype(np.float64)
    rel = (got - ref) / ref
    assert np.abs(rel).max() <= 2.0 ** -24 + 2.0 ** -30  # the final rounding to FP32
    assert abs(float(rel.mean())) < 2.0 ** -30


def test_gemm_f32_sliced_zero_tiny_rows_and_k0(cuda_lib):
    lib = cuda_lib.load()
    g = np.random.default_rng(29)
    A = g.standard_normal((150, 48)).astype(np.float32)
    B = g.standard_normal((48, 70)).astype(np.float32)
    A[3] = 0.0
    A[5] *= np.float32(2.0 ** -100)   # tiny but above the 2^-118 cut: kept
    A[7, :32] = 1e-37                 # below the cut in the first K block: counts as zero there
    got = _gemm(lib, A, B, np.zeros((150, 70), np.float32), fn="tt_gemm_f32_sliced")
    ref = A.astype(np.float64) @ B.astype(np.float64)
    assert np.all(got[3] == 0.0)
    assert np.allclose(got[5], ref[5], rtol=0, atol=2.0 ** -100 * 1e-5)
    ok = np.ones(150, bool)
    ok[[3, 5, 7]] = False
    assert np.all(np.abs(got[ok] - ref[ok]) <= _sliced_bound(A, B)[ok] + 2.0 ** -24 * np.abs(ref[ok]))
    assert np.abs(got[7] - ref[7]).max() <= 1e-35 + np.abs(ref[7]).max() * 1e-6
    # K = 0: C <- beta C
    C0 = g.standard_normal((40, 30)).astype(np.float32)
    got0 = _gemm(lib, np.zeros((40, 0), np.float32), np.zeros((0, 30), np.float32), C0.copy(), 1.0, 2.0,
                 fn="tt_gemm_f32_sliced")
    assert np.array_equal(got0, 2.0 * C0)


def test_gemm_f32_sliced_twice_identical(cuda_lib):
    lib = cuda_lib.load()
    g = np.random.default_rng(31)
    A = g.standard_normal((500, 300)).astype(np.float32)
    B = g.standard_normal((300, 260)).astype(np.float32)
    a = _gemm(lib, A, B, np.zeros((500, 260), np.float32), fn="tt_gemm_f32_sliced")
    b = _gemm(lib, A, B, np.zeros((500, 260), np.float32), fn="tt_gemm_f32_sliced")
    assert np.array_equal(a, b)
