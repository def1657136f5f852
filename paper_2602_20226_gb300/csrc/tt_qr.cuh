// Householder QR used by the rounding sweeps.
#pragma once

#include <vector>

#include "tt_common.cuh"
#include "tt_gemm.cuh"

namespace tt {

// Scratch of one QR (all device memory, carved from the caller's workspace).
template <typename T>
struct QrWork {
  int nb = 16;       // panel width (<= 32)
  T* tau = nullptr;  // [>= min(m, n)]
  T* tmat = nullptr; // [npanels][nb][nb] T factors (column-major)
  double* tmat64 = nullptr;  // FP32 matrices: the T factors in FP64 (recomputed from the
                             // FP32-rounded reflectors), [npanels][nb][nb]
  T* vbuf = nullptr; // explicit Householder vectors, column-major, ld = ldv >= m
  int ldv = 0;
  T* w1 = nullptr;   // [nb * ncols]
  T* w2 = nullptr;   // [nb * ncols]
  unsigned* status = nullptr;  // device word: ST_TIMEOUT if a tensor-core GEMM's wait expired
  // filled by householder_qr
  int m = 0, n = 0, npanels = 0;
};

// In-place QR of the column-major m x n matrix A (ld lda): on return the upper
// trapezoid holds R (min(m,n) x n) and w holds the reflectors.
template <typename T>
int householder_qr(cudaStream_t s, T* A, int m, int n, int lda, QrWork<T>& w);

// Thin Q (m x min(m,n), column-major, ld ldq) from the reflectors of the last QR.
template <typename T>
int form_thin_q(cudaStream_t s, const QrWork<T>& w, T* Q, int ldq);

// ---- batched forms: one job per train of a batch, the panels of all jobs in lock-step
template <typename T>
struct QrJob {
  T* A;  // m x n, column-major, ld lda: QR'd in place
  int m, n, lda;
  T* tau;
  T* tmat;  // T factors, [panel][nb][nb]
  T* vbuf;  // explicit reflectors, ld ldv
  int ldv;
  T* w1;    // [nb * max(n, min(m, n))]
  T* w2;    // [nb * max(n, min(m, n))]
  T* Q;     // form_thin_q_batched: m x min(m, n), ld ldq
  int ldq;
  // FP32 jobs (the mixed form): the T factors in FP64, [panel][nb][nb], recomputed from the
  // FP32-rounded reflectors by the FP64 panel kernel, and W1 = V^T X, W2 = op(T) W1 in FP64
  // ([nb * max(n, min(m, n))] each) for the updates X -= V W2.
  double* tmat64 = nullptr;
  double* w1d = nullptr;
  double* w2d = nullptr;
};

// hj: the jobs on the host (sizes, for the launch shapes and the update GEMMs);
// d_jobs: the same array in device memory; status (may be null): raises ST_TIMEOUT if a
// tensor-core GEMM's wait expired.
template <typename T>
int householder_qr_batched(cudaStream_t s, const std::vector<QrJob<T>>& hj, const QrJob<T>* d_jobs, int nb,
                           JobArena& arena, unsigned* status = nullptr);
template <typename T>
int form_thin_q_batched(cudaStream_t s, const std::vector<QrJob<T>>& hj, const QrJob<T>* d_jobs, int nb,
                        JobArena& arena, unsigned* status = nullptr);

}  // namespace tt
