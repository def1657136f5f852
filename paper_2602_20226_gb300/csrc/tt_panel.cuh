// Householder panel factorisation and block-reflector application (tt_panel.cu).
#pragma once

#include "tt_common.cuh"

namespace tt {

// Householder QR of the panel of jb <= nb columns at column (and row) j0 of the column-major
// matrix A (m rows, ld lda), in FP64 arithmetic.  On return A holds R (upper part of the panel)
// and the reflector entries below the diagonal, Vb (ld ldv) the explicit unit-lower reflectors,
// Tm (FP64, ld ldt) the upper-triangular T of the compact form I - V T V^T, tau the scalars.
// TIO = double: the plain FP64 form.  TIO = float: the mixed form; A and Vb receive the result
// rounded to FP32 and tau / T are recomputed in FP64 from the ROUNDED reflectors, so that
// I - V T V^T is orthogonal (to FP64 rounding) for the V that the FP32 updates use.
// Panels of at least 256 rows are spread over an 8-CTA cluster.  nb = 16 or 32.
template <typename TIO>
int qr_panel_fast(cudaStream_t s, TIO* A, int lda, int m, int j0, int jb, int nb, TIO* tau, double* Tm,
                  int ldt, TIO* Vb, int ldv);

// X <- (I - V op(T) V^T) X for the mr x nc column-major block X (ld ldx) and the jb explicit
// reflectors V (mr x jb, ld ldv): op(T) = T^T applies Q^T (the QR's trailing update),
// op(T) = T applies Q (forming the thin Q).  One launch: W1 = V^T X, W2 = op(T) W1 and the
// update X -= V W2 per block of columns.  T = double: FP64.  T = float: W1 by compensated
// FP32 dot products (Dot2; the reflectors and X are FP32, so the products are exact), W1 and
// W2 kept in FP64, and V W2 summed in float-float before the single rounding of X to FP32.
template <typename T>
int apply_block_reflector(cudaStream_t s, const T* V, int ldv, int mr, int jb, const double* Tm, int ldt,
                          bool transpose_t, T* X, int ldx, int nc);

// Batched form of qr_panel_fast: the panel at column j0 of every job (one CTA per job).
struct PanelJob {
  void* A;        // column-major m x n (TIO), ld lda
  int m, n, lda;
  void* tau;      // TIO [>= min(m, n)]
  double* Tm;     // FP64 T factors, [panel][nb][nb]
  void* Vb;       // explicit reflectors (TIO), ld ldv
  int ldv;
};
template <typename TIO>
int qr_panel_fast_batched(cudaStream_t s, int njobs, const PanelJob* d_jobs, int j0, int nb, int mr_max);

}  // namespace tt
