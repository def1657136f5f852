// Core-by-core exact operations (Section 3.1) and the small reshaping kernels of
// the rounding sweeps.
//
// apply / hadamard write every core of the result in ONE launch: a warp owns one
// output row (a, r, i) of one site and streams the contiguous (a', r') columns, so
// the write (the dominant HBM traffic, a*a' or r*s times the input) is coalesced and
// the index arithmetic is paid once per row, not per element.
#include "tt_kernels.cuh"

namespace tt {

namespace {

template <typename T>
__device__ __forceinline__ int find_site(const long long* start, int L, long long row) {
  int lo = 0, hi = L;  // start[lo] <= row < start[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (start[mid] <= row) lo = mid; else hi = mid;
  }
  return lo;
}

// Y_k[(a, r), i, (a', r')] = sum_j W_k[a, i, j, a'] G_k[r, j, r']
template <typename T>
__global__ void __launch_bounds__(256) apply_kernel(ApplyParams<T> P) {
  const long long row = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= P.row_start[P.L]) return;
  const int k = find_site<T>(P.row_start, P.L, row);
  const ApplySite<T>& S = P.site[k];
  const long long local = row - P.row_start[k];
  const int d = S.d, a1 = S.a1, r0 = S.r0, r1 = S.r1;
  const int i = (int)(local % d);
  const long long t = local / d;
  const int r = (int)(t % r0);
  const int a = (int)(t / r0);
  T* out = S.y + local * (long long)a1 * r1;
  const T* wrow = S.w + (long long)(a * d + i) * d * a1;  // W[a, i, :, :]
  for (int ap = 0; ap < a1; ++ap) {
    for (int rp = lane; rp < r1; rp += 32) {
      T acc = T(0);
      for (int j = 0; j < d; ++j)
        acc += wrow[(long long)j * a1 + ap] * S.g[((long long)r * d + j) * r1 + rp];
      out[(long long)ap * r1 + rp] = acc;
    }
  }
}

// Z_k[(r, s), i, (r', s')] = X_k[r, i, r'] Y_k[s, i, s']
template <typename T>
__global__ void __launch_bounds__(256) hadamard_kernel(HadamardParams<T> P) {
  const long long row = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= P.row_start[P.L]) return;
  const int k = find_site<T>(P.row_start, P.L, row);
  const HadamardSite<T>& S = P.site[k];
  const long long local = row - P.row_start[k];
  const int d = S.d, r1 = S.r1, s0 = S.s0, s1 = S.s1;
  const int i = (int)(local % d);
  const long long t = local / d;
  const int s = (int)(t % s0);
  const int r = (int)(t / s0);
  T* out = S.z + local * (long long)r1 * s1;
  const T* xrow = S.x + ((long long)r * d + i) * r1;
  const T* yrow = S.y + ((long long)s * d + i) * s1;
  for (int rp = 0; rp < r1; ++rp) {
    const T xv = xrow[rp];
    for (int sp = lane; sp < s1; sp += 32) out[(long long)rp * s1 + sp] = xv * yrow[sp];
  }
}

// dG_k[r, j, r'] += sum_{a, a', i} W_k[a, i, j, a'] dY_k[(a, r), i, (a', r')]
// one warp per (r, j) row of dG
template <typename T>
__global__ void __launch_bounds__(256) apply_bwd_x_kernel(ApplyBwdParams<T> P) {
  const long long row = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= P.row_start[P.L]) return;
  const int k = find_site<T>(P.row_start, P.L, row);
  const ApplyBwdSite<T>& S = P.site[k];
  const long long local = row - P.row_start[k];
  const int d = S.d, a0 = S.a0, a1 = S.a1, r0 = S.r0, r1 = S.r1;
  const int j = (int)(local % d);
  const int r = (int)(local / d);
  T* out = S.dg + local * r1;
  for (int rp = lane; rp < r1; rp += 32) {
    T acc = T(0);
    for (int a = 0; a < a0; ++a)
      for (int i = 0; i < d; ++i) {
        const T* dyrow = S.dy + (((long long)a * r0 + r) * d + i) * ((long long)a1 * r1);
        const T* w = S.w + ((long long)(a * d + i) * d + j) * a1;
        for (int ap = 0; ap < a1; ++ap) acc += w[ap] * dyrow[(long long)ap * r1 + rp];
      }
    out[rp] += acc;
  }
}

// dW_k[a, i, j, a'] += sum_{r, r'} G_k[r, j, r'] dY_k[(a, r), i, (a', r')]
// one CTA per (site, a, i, a'); all d values of j at once
template <typename T>
__global__ void __launch_bounds__(256) apply_bwd_w_kernel(ApplyBwdParams<T> P) {
  __shared__ double red[TT_MAX_MODE][8];
  const long long blk = blockIdx.x;
  if (blk >= P.wblk_start[P.L]) return;
  const int k = find_site<T>(P.wblk_start, P.L, blk);
  const ApplyBwdSite<T>& S = P.site[k];
  const long long local = blk - P.wblk_start[k];
  const int d = S.d, a0 = S.a0, a1 = S.a1, r0 = S.r0, r1 = S.r1;
  const int ap = (int)(local % a1);
  const long long t = local / a1;
  const int i = (int)(t % d);
  const int a = (int)(t / d);
  (void)a0;
  double acc[TT_MAX_MODE];
  for (int j = 0; j < d; ++j) acc[j] = 0.0;
  const long long n = (long long)r0 * r1;
  for (long long e = threadIdx.x; e < n; e += blockDim.x) {
    const int r = (int)(e / r1), rp = (int)(e % r1);
    const double dy = (double)S.dy[(((long long)a * r0 + r) * d + i) * ((long long)a1 * r1) +
                                   (long long)ap * r1 + rp];
    for (int j = 0; j < d; ++j) acc[j] += dy * (double)S.g[((long long)r * d + j) * r1 + rp];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = 0; j < d; ++j) {
    double v = warp_sum(acc[j]);
    if (lane == 0) red[j][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < d) {
    double v = 0.0;
    for (int w = 0; w < 8; ++w) v += red[threadIdx.x][w];
    const int j = threadIdx.x;
    T* p = S.dw + (((long long)a * d + i) * d + j) * a1 + ap;
    *p += (T)v;
  }
}

// dX_k[r, i, r'] += sum_{s, s'} dZ_k[(r, s), i, (r', s')] Y_k[s, i, s']  (warp per (r, i, r'))
template <typename T>
__global__ void __launch_bounds__(256) hadamard_bwd_x_kernel(HadamardBwdParams<T> P) {
  const long long row = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= P.xrow_start[P.L]) return;
  const int k = find_site<T>(P.xrow_start, P.L, row);
  const HadamardBwdSite<T>& S = P.site[k];
  const long long local = row - P.xrow_start[k];
  const int d = S.d, r0 = S.r0, r1 = S.r1, s0 = S.s0, s1 = S.s1;
  (void)r0;
  const int rp = (int)(local % r1);
  const long long t = local / r1;
  const int i = (int)(t % d);
  const int r = (int)(t / d);
  double acc = 0.0;
  for (int s = 0; s < s0; ++s) {
    const T* dz = S.dz + (((long long)r * s0 + s) * d + i) * ((long long)r1 * s1) + (long long)rp * s1;
    const T* y = S.y + ((long long)s * d + i) * s1;
    for (int sp = lane; sp < s1; sp += 32) acc += (double)dz[sp] * (double)y[sp];
  }
  acc = warp_sum(acc);
  if (lane == 0) S.dx[((long long)r * d + i) * r1 + rp] += (T)acc;
}

// dY_k[s, i, s'] += sum_{r, r'} dZ_k[(r, s), i, (r', s')] X_k[r, i, r']  (warp per (s, i))
template <typename T>
__global__ void __launch_bounds__(256) hadamard_bwd_y_kernel(HadamardBwdParams<T> P) {
  const long long row = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= P.yrow_start[P.L]) return;
  const int k = find_site<T>(P.yrow_start, P.L, row);
  const HadamardBwdSite<T>& S = P.site[k];
  const long long local = row - P.yrow_start[k];
  const int d = S.d, r0 = S.r0, r1 = S.r1, s0 = S.s0, s1 = S.s1;
  const int i = (int)(local % d);
  const int s = (int)(local / d);
  T* out = S.dy + ((long long)s * d + i) * s1;
  for (int sp = lane; sp < s1; sp += 32) {
    double acc = 0.0;
    for (int r = 0; r < r0; ++r) {
      const T* dz = S.dz + (((long long)r * s0 + s) * d + i) * ((long long)r1 * s1) + sp;
      const T* x = S.x + ((long long)r * d + i) * r1;
      for (int rp = 0; rp < r1; ++rp) acc += (double)dz[(long long)rp * s1] * (double)x[rp];
    }
    out[sp] += (T)acc;
  }
}

// row-major (m x n) -> column-major (m x n), i.e. an out-of-place transpose
template <typename T>
__global__ void transpose_kernel(const T* __restrict__ src, int m, int n, T* __restrict__ dst) {
  __shared__ T tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int yy = threadIdx.y; yy < 32; yy += 8) {
    const int i = by + yy, j = bx + threadIdx.x;
    if (i < m && j < n) tile[yy][threadIdx.x] = src[(long long)i * n + j];
  }
  __syncthreads();
  for (int yy = threadIdx.y; yy < 32; yy += 8) {
    const int j = bx + yy, i = by + threadIdx.x;
    if (i < m && j < n) dst[(long long)j * m + i] = tile[threadIdx.x][yy];
  }
}

// Rbuf (p x n, column-major, zeros below the diagonal) from the QR'd A (ld lda)
template <typename T>
__global__ void extract_r_kernel(const T* A, int lda, int p, int n, T* R) {
  const long long total = (long long)p * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % p), c = (int)(e / p);
    R[e] = (i <= c) ? A[i + (long long)c * lda] : T(0);
  }
}

// X = R (p x n, column-major, FP64, zeros below the diagonal) from the QR'd A (ld lda)
template <typename T>
__global__ void extract_r_f64_kernel(const T* A, int lda, int p, int n, double* X) {
  const long long total = (long long)p * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % p), c = (int)(e / p);
    X[e] = (i <= c) ? (double)A[i + (long long)c * lda] : 0.0;
  }
}

// X = R^T (n x p, column-major, FP64) from the QR'd A (ld lda)
template <typename T>
__global__ void extract_rt_kernel(const T* A, int lda, int p, int n, double* X) {
  const long long total = (long long)p * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e % n), i = (int)(e / n);  // X[c + i*n] = R[i][c]
    X[e] = (i <= c) ? (double)A[i + (long long)c * lda] : 0.0;
  }
}

template <typename T>
__global__ void __launch_bounds__(1024) sumsq_kernel(const T* a, long long n, double* out) {
  __shared__ double scratch[32];
  double s = 0.0;
  for (long long e = threadIdx.x; e < n; e += blockDim.x) {
    const double v = (double)a[e];
    s = fma(v, v, s);
  }
  s = block_sum(s, scratch);
  if (threadIdx.x == 0) *out = sqrt(s);
}

__global__ void f64_to_f32_kernel(const double* a, long long n, float* b) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    b[e] = (float)a[e];
}

__global__ void f32_to_f64_kernel(const float* a, long long n, double* b) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    b[e] = (double)a[e];
}

// G <- 1.5 I - 0.5 G  (n x n, column-major): the Newton-Schulz factor for U^T U = G
__global__ void ns_h_kernel(float* G, int n) {
  const long long total = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), c = (int)(e / n);
    G[e] = (i == c ? 1.5f : 0.0f) - 0.5f * G[e];
  }
}

inline int grid_for(long long total, int per_block, int cap = 1 << 20) {
  return (int)std::max<long long>(1, std::min<long long>(ceil_div(total, per_block), cap));
}

}  // namespace

template <typename T>
int launch_apply(cudaStream_t s, const ApplyParams<T>& P) {
  const long long rows = P.row_start[P.L];
  if (rows == 0) return TT_OK;
  if (ceil_div(rows, 8) > 0x7fffffffLL) return fail(TT_ERR_UNSUPPORTED, "apply: too many rows");
  apply_kernel<T><<<(unsigned)ceil_div(rows, 8), 256, 0, s>>>(P);
  TT_LAUNCH_CHECK();
  return TT_OK;
}

template <typename T>
int launch_hadamard(cudaStream_t s, const HadamardParams<T>& P) {
  const long long rows = P.row_start[P.L];
  if (rows == 0) return TT_OK;
  if (ceil_div(rows, 8) > 0x7fffffffLL) return fail(TT_ERR_UNSUPPORTED, "hadamard: too many rows");
  hadamard_kernel<T><<<(unsigned)ceil_div(rows, 8), 256, 0, s>>>(P);
  TT_LAUNCH_CHECK();
  return TT_OK;
}

template <typename T>
int launch_apply_bwd(cudaStream_t s, const ApplyBwdParams<T>& P, bool want_x, bool want_w) {
  if (want_x && P.row_start[P.L] > 0) {
    apply_bwd_x_kernel<T><<<(unsigned)ceil_div(P.row_start[P.L], 8), 256, 0, s>>>(P);
    TT_LAUNCH_CHECK();
  }
  if (want_w && P.wblk_start[P.L] > 0) {
    apply_bwd_w_kernel<T><<<(unsigned)P.wblk_start[P.L], 256, 0, s>>>(P);
    TT_LAUNCH_CHECK();
  }
  return TT_OK;
}

template <typename T>
int launch_hadamard_bwd(cudaStream_t s, const HadamardBwdParams<T>& P, bool want_x, bool want_y) {
  if (want_x && P.xrow_start[P.L] > 0) {
    hadamard_bwd_x_kernel<T><<<(unsigned)ceil_div(P.xrow_start[P.L], 8), 256, 0, s>>>(P);
    TT_LAUNCH_CHECK();
  }
  if (want_y && P.yrow_start[P.L] > 0) {
    hadamard_bwd_y_kernel<T><<<(unsigned)ceil_div(P.yrow_start[P.L], 8), 256, 0, s>>>(P);
    TT_LAUNCH_CHECK();
  }
  return TT_OK;
}

template <typename T>
int transpose_rm_to_cm(cudaStream_t s, const T* src, int m, int n, T* dst) {
  if (m <= 0 || n <= 0) return TT_OK;
  dim3 grid((unsigned)ceil_div(n, 32), (unsigned)ceil_div(m, 32));
  transpose_kernel<T><<<grid, dim3(32, 8), 0, s>>>(src, m, n, dst);
  TT_LAUNCH_CHECK();
  return TT_OK;
}

template <typename T>
int extract_r(cudaStream_t s, const T* A, int lda, int p, int n, T* R) {
  extract_r_kernel<T><<<grid_for((long long)p * n, 256, 4096), 256, 0, s>>>(A, lda, p, n, R);
  TT_LAUNCH_CHECK();
  return TT_OK;
}

template <typename T>
int extract_r_f64(cudaStream_t s, const T* A, int lda, int p, int n, double* X) {
  extract_r_f64_kernel<T><<<grid_for((long long)p * n, 256, 4096), 256, 0, s>>>(A, lda, p, n, X);
  TT_LAUNCH_CHECK();
  return TT_OK;
}

template <typename T>
int extract_rt(cudaStream_t s, const T* A, int lda, int p, int n, double* X) {
  extract_rt_kernel<T><<<grid_for((long long)p * n, 256, 4096), 256, 0, s>>>(A, lda, p, n, X);
  TT_LAUNCH_CHECK();
  return TT_OK;
}

template <typename T>
int copy_matrix(cudaStream_t s, const T* src, int p, int n, T* dst) {
  TT_CUDA_CHECK(cudaMemcpyAsync(dst, src, (size_t)p * n * sizeof(T), cudaMemcpyDeviceToDevice, s));
  return TT_OK;
}

template <typename T>
int frobenius_norm(cudaStream_t s, const T* a, long long n, double* out) {
  sumsq_kernel<T><<<1, 1024, 0, s>>>(a, n, out);
  TT_LAUNCH_CHECK();
  return TT_OK;
}

int convert_f64_to_f32(cudaStream_t s, const double* a, long long n, float* b) {
  f64_to_f32_kernel<<<grid_for(n, 256, 4096), 256, 0, s>>>(a, n, b);
  TT_LAUNCH_CHECK();
  return TT_OK;
}

int convert_f32_to_f64(cudaStream_t s, const float* a, long long n, double* b) {
  f32_to_f64_kernel<<<grid_for(n, 256, 4096), 256, 0, s>>>(a, n, b);
  TT_LAUNCH_CHECK();
  return TT_OK;
}

int newton_schulz_h(cudaStream_t s, float* G, int n) {
  ns_h_kernel<<<grid_for((long long)n * n, 256, 4096), 256, 0, s>>>(G, n);
  TT_LAUNCH_CHECK();
  return TT_OK;
}

#define TT_EW_INST(T)                                                                   \
  template int launch_apply<T>(cudaStream_t, const ApplyParams<T>&);                    \
  template int launch_hadamard<T>(cudaStream_t, const HadamardParams<T>&);              \
  template int launch_apply_bwd<T>(cudaStream_t, const ApplyBwdParams<T>&, bool, bool); \
  template int launch_hadamard_bwd<T>(cudaStream_t, const HadamardBwdParams<T>&, bool, bool); \
  template int transpose_rm_to_cm<T>(cudaStream_t, const T*, int, int, T*);             \
  template int extract_r<T>(cudaStream_t, const T*, int, int, int, T*);                 \
  template int extract_rt<T>(cudaStream_t, const T*, int, int, int, double*);           \
  template int extract_r_f64<T>(cudaStream_t, const T*, int, int, int, double*);        \
  template int frobenius_norm<T>(cudaStream_t, const T*, long long, double*);           \
  template int copy_matrix<T>(cudaStream_t, const T*, int, int, T*);
TT_EW_INST(double)
TT_EW_INST(float)
#undef TT_EW_INST

}  // namespace tt
