// Launch descriptors and launchers of the core-by-core kernels.
#pragma once

#include <algorithm>

#include "tt_common.cuh"

namespace tt {

template <typename T>
struct ApplySite {
  const T* w;
  const T* g;
  T* y;
  int d, a0, a1, r0, r1;
};
template <typename T>
struct ApplyParams {
  int L;
  long long row_start[TT_MAX_SITES + 1];  // warp rows (a, r, i) per site, prefix sums
  ApplySite<T> site[TT_MAX_SITES];
};

template <typename T>
struct HadamardSite {
  const T* x;
  const T* y;
  T* z;
  int d, r0, r1, s0, s1;
};
template <typename T>
struct HadamardParams {
  int L;
  long long row_start[TT_MAX_SITES + 1];  // rows (r, s, i)
  HadamardSite<T> site[TT_MAX_SITES];
};

template <typename T>
struct ApplyBwdSite {
  const T* w;
  const T* g;
  const T* dy;
  T* dg;
  T* dw;
  int d, a0, a1, r0, r1;
};
template <typename T>
struct ApplyBwdParams {
  int L;
  long long row_start[TT_MAX_SITES + 1];   // rows (r, j) of dG
  long long wblk_start[TT_MAX_SITES + 1];  // CTAs (a, i, a') for dW
  ApplyBwdSite<T> site[TT_MAX_SITES];
};

template <typename T>
struct HadamardBwdSite {
  const T* x;
  const T* y;
  const T* dz;
  T* dx;
  T* dy;
  int d, r0, r1, s0, s1;
};
template <typename T>
struct HadamardBwdParams {
  int L;
  long long xrow_start[TT_MAX_SITES + 1];  // rows (r, i, r') of dX
  long long yrow_start[TT_MAX_SITES + 1];  // rows (s, i) of dY
  HadamardBwdSite<T> site[TT_MAX_SITES];
};

template <typename T>
int launch_apply(cudaStream_t s, const ApplyParams<T>& P);
template <typename T>
int launch_hadamard(cudaStream_t s, const HadamardParams<T>& P);
template <typename T>
int launch_apply_bwd(cudaStream_t s, const ApplyBwdParams<T>& P, bool want_x, bool want_w);
template <typename T>
int launch_hadamard_bwd(cudaStream_t s, const HadamardBwdParams<T>& P, bool want_x, bool want_y);

template <typename T>
int transpose_rm_to_cm(cudaStream_t s, const T* src, int m, int n, T* dst);
template <typename T>
int extract_r(cudaStream_t s, const T* A, int lda, int p, int n, T* R);
template <typename T>
int extract_rt(cudaStream_t s, const T* A, int lda, int p, int n, double* X);
template <typename T>
int extract_r_f64(cudaStream_t s, const T* A, int lda, int p, int n, double* X);
template <typename T>
int frobenius_norm(cudaStream_t s, const T* a, long long n, double* out);
template <typename T>
int copy_matrix(cudaStream_t s, const T* src, int p, int n, T* dst);

int convert_f64_to_f32(cudaStream_t s, const double* a, long long n, float* b);
int convert_f32_to_f64(cudaStream_t s, const float* a, long long n, double* b);

// ---- batched maps (tt_batch_ops.cu): dst(i, j) = op(src(i, j)) for i < rows, j < cols,
// src(i, j) = src[i sr + j sc], dst(i, j) = dst[i dr + j dc]; one job per train.
enum MapOp : int {
  MAP_COPY = 0,
  MAP_UPPER = 1,  // zero below the diagonal (i > j)
  MAP_NS = 2      // 1.5 [i == j] - 0.5 src (the Newton-Schulz factor)
};
struct MapJob {
  const void* src;
  void* dst;
  int rows, cols;
  int64_t sr, sc, dr, dc;
  int op;
};
template <typename TS, typename TD>
int map_batched(cudaStream_t s, int nj, const MapJob* d_jobs, int64_t max_elems);

struct NormJob {
  const void* src;  // n contiguous values
  int64_t n;
  double* out;      // ||src||_2 in FP64
};
template <typename T>
int norm_batched(cudaStream_t s, int nj, const NormJob* d_jobs);
int newton_schulz_h(cudaStream_t s, float* G, int n);  // G <- 1.5 I - 0.5 G

}  // namespace tt
