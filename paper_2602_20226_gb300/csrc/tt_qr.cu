// Blocked Householder QR of a column-major m x n matrix (used by both rounding sweeps).
//
// Panel of nb columns: one CTA factors it column by column (Householder vector,
// tau, and the upper-triangular T of the compact WY form I - V T V^T), reading the
// panel from global memory.  For every column the dot products of the new
// Householder vector with all other panel columns (the trailing-column update and
// the column of T) come out of ONE block reduction: a 32-wide warp reduce-scatter
// followed by a cross-warp sum in shared memory.
//
// Trailing update A <- (I - V T^T V^T) A and thin-Q formation
// Q = H_1 ... H_p [I; 0] take two launches per panel: W2 = op(T) V^T A (one CTA per
// column, a reduction over the rows) and the rank-nb update A -= V W2 (the GEMM of
// the form: FP64 SIMT, or tensor cores for FP32).
#include <cooperative_groups.h>

#include <type_traits>

#include "tt_kernels.cuh"
#include "tt_qr.cuh"

namespace cg = cooperative_groups;

namespace tt {

namespace {

template <typename T, int NT>
__device__ __forceinline__ void panel_body(T* __restrict__ A, int lda, int m, int j0, int jb,
                                           T* __restrict__ tau, T* __restrict__ Tm, int ldt,
                                           T* __restrict__ Vb, int ldv, bool staged) {
  constexpr int NW = NT / 32;
  extern __shared__ unsigned char panel_raw[];
  __shared__ T red[NW][33];
  __shared__ T dvec[32];
  __shared__ T Ts[32][33];
  __shared__ T s_tau, s_scal;
  __shared__ T s_sum[32];
  __shared__ int s_nz;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int mr = m - j0;
  // the panel (rows j0..m-1, columns j0..j0+jb-1): in shared memory when it fits,
  // column c at P + c*mr (row i at index i - j0), else read in place
  T* P = reinterpret_cast<T*>(panel_raw);
  auto col = [&](int c) -> T* { return staged ? (P + (int64_t)c * mr - j0) : (A + (int64_t)(j0 + c) * lda); };
  const int64_t ld_panel = staged ? (int64_t)mr : (int64_t)lda;
  if (staged) {
    for (int c = 0; c < jb; ++c) {
      const T* src = A + (int64_t)(j0 + c) * lda;
      for (int i = j0 + tid; i < m; i += NT) P[(int64_t)c * mr + (i - j0)] = src[i];
    }
  }
  for (int e = tid; e < 32 * 33; e += NT) (&Ts[0][0])[e] = T(0);
  __syncthreads();

  for (int c = 0; c < jb; ++c) {
    const int j = j0 + c;
    T* colj = col(c);
    // ---- 1. norm of the part below the diagonal
    T part = T(0);
    for (int i = j + 1 + tid; i < m; i += NT) {
      const T v = colj[i];
      part += v * v;
    }
    const T s = block_sum(part, s_sum);
    if (tid == 0) {
      const T alpha = colj[j];
      if (s == T(0)) {
        s_tau = T(0);
        s_scal = T(1);
        s_nz = 0;
      } else {
        const T beta = -copysign(sqrt(alpha * alpha + s), alpha);
        s_tau = (beta - alpha) / beta;
        s_scal = T(1) / (alpha - beta);
        colj[j] = beta;
        s_nz = 1;
      }
    }
    __syncthreads();
    const T tj = s_tau;
    if (s_nz) {
      const T sc = s_scal;
      for (int i = j + 1 + tid; i < m; i += NT) colj[i] *= sc;
    }
    __syncthreads();
    // ---- 2. d_t = A[j, j0+t] + sum_{i>j} A[i, j] A[i, j0+t]  for every t != c
    //      (t < c: v_t^T v_c for the T factor; t > c: v_c^T a_t for the update)
    T acc[32];
#pragma unroll
    for (int t = 0; t < 32; ++t) acc[t] = T(0);
    const T* c0 = col(0);
    for (int i = j + 1 + tid; i < m; i += NT) {
      const T vi = colj[i];
#pragma unroll
      for (int t = 0; t < 32; ++t)
        if (t < jb) acc[t] += vi * c0[(int64_t)t * ld_panel + i];
    }
    warp_reduce_scatter32(acc, lane);
    red[warp][lane] = acc[0];
    __syncthreads();
    if (tid < 32) {
      T d = T(0);
#pragma unroll
      for (int w = 0; w < NW; ++w) d += red[w][tid];
      if (tid < jb) d += col(tid)[j];
      dvec[tid] = d;
    }
    __syncthreads();
    // ---- 3. apply H_c to the remaining panel columns, and extend T
    if (tj != T(0)) {
      for (int t = c + 1; t < jb; ++t) {
        const T f = tj * dvec[t];
        T* colt = col(t);
        for (int i = j + 1 + tid; i < m; i += NT) colt[i] -= f * colj[i];
      }
      if (tid > c && tid < jb) col(tid)[j] -= tj * dvec[tid];
    }
    if (tid < c) {
      T v = T(0);
      for (int q = tid; q < c; ++q) v += Ts[tid][q] * dvec[q];
      Ts[tid][c] = -tj * v;
    }
    if (tid == 0) {
      Ts[c][c] = tj;
      tau[j] = tj;
    }
    __syncthreads();
  }
  // write back the factored panel (R above, reflectors below), the explicit
  // unit-lower-trapezoidal V (rows j0..m-1) and T
  for (int t = 0; t < jb; ++t) {
    const int jc = j0 + t;
    const T* src = col(t);
    T* dstA = A + (int64_t)jc * lda;
    T* dst = Vb + (int64_t)jc * ldv;
    for (int i = j0 + tid; i < m; i += NT) {
      const T v = src[i];
      if (staged) dstA[i] = v;
      dst[i] = (i < jc) ? T(0) : (i == jc ? T(1) : v);
    }
  }
  for (int e = tid; e < jb * jb; e += NT) {
    const int r = e % jb, cc = e / jb;
    Tm[r + (int64_t)cc * ldt] = Ts[r][cc];
  }
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT) qr_panel_kernel(T* __restrict__ A, int lda, int m, int j0,
                                                      int jb, T* __restrict__ tau,
                                                      T* __restrict__ Tm, int ldt,
                                                      T* __restrict__ Vb, int ldv, bool staged) {
  panel_body<T, NT>(A, lda, m, j0, jb, tau, Tm, ldt, Vb, ldv, staged);
}

// Batched: the panel at column j0 of every job (one CTA per job), staged in shared
// memory when mr x jb fits in smem_cap bytes.
template <typename T, int NT>
__global__ void __launch_bounds__(NT) qr_panel_batched_kernel(const QrJob<T>* __restrict__ jobs, int j0,
                                                              int nb, size_t smem_cap) {
  const QrJob<T> J = jobs[blockIdx.x];
  const int p = min(J.m, J.n);
  if (j0 >= p) return;
  const int jb = min(nb, p - j0);
  const bool staged = (size_t)(J.m - j0) * jb * sizeof(T) <= smem_cap;
  panel_body<T, NT>(J.A, J.lda, J.m, j0, jb, J.tau, J.tmat + (int64_t)(j0 / nb) * nb * nb, nb, J.vbuf, J.ldv,
                    staged);
}

// The same panel factorisation spread over a thread-block cluster of CS CTAs: CTA c
// keeps rows [c*chunk, (c+1)*chunk) of the panel in its shared memory; for every
// column the partial norms and the partial dot products of the new reflector with
// the other panel columns are combined through distributed shared memory, with two
// cluster barriers per column (partials are double-buffered by column parity, so a
// slot is rewritten only after every CTA has passed the next barrier).  CS SMs share
// the panel's arithmetic, which matters most in FP64.
template <typename T, int NT, int CS>
__global__ void __launch_bounds__(NT) qr_panel_cluster_kernel(T* __restrict__ A, int lda, int m, int j0,
                                                              int jb, T* __restrict__ tau,
                                                              T* __restrict__ Tm, int ldt,
                                                              T* __restrict__ Vb, int ldv, int chunk) {
  constexpr int NW = NT / 32;
  extern __shared__ unsigned char panel_raw[];
  __shared__ T red[NW][33];
  __shared__ T Ts[32][33];
  __shared__ T s_sum[32];
  __shared__ T norm_part[2], alpha_slot[2];
  __shared__ T dot_part[2][32];
  __shared__ T dvec[32];
  __shared__ T s_tau, s_scal;
  __shared__ int s_nz;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int mr = m - j0;
  const int lo = min(mr, rank * chunk), hi = min(mr, (rank + 1) * chunk);  // local panel rows
  T* P = reinterpret_cast<T*>(panel_raw);  // column c at P + c*chunk, local row l at index l - lo
  auto at = [&](int c, int l) -> T& { return P[(int64_t)c * chunk + (l - lo)]; };
  for (int c = 0; c < jb; ++c) {
    const T* src = A + (int64_t)(j0 + c) * lda + j0;
    for (int l = lo + tid; l < hi; l += NT) at(c, l) = src[l];
  }
  for (int e = tid; e < 32 * 33; e += NT) (&Ts[0][0])[e] = T(0);
  __syncthreads();

  for (int c = 0; c < jb; ++c) {
    const int b = c & 1;
    const int jl = c;  // local row of the diagonal element
    const bool own = (jl >= lo && jl < hi);
    const int r0 = max(lo, jl + 1);  // first own row below the diagonal
    // ---- 1. partial norm below the diagonal
    T part = T(0);
    for (int l = r0 + tid; l < hi; l += NT) {
      const T v = at(c, l);
      part += v * v;
    }
    part = block_sum(part, s_sum);
    if (tid == 0) {
      norm_part[b] = part;
      if (own) alpha_slot[b] = at(c, jl);
    }
    cluster_sync_all();
    if (tid == 0) {
      T sum = T(0);
      for (int r = 0; r < CS; ++r) sum += dsmem_load(&norm_part[b], r);
      const int owner = jl / chunk;
      const T alpha = dsmem_load(&alpha_slot[b], owner);
      if (sum == T(0)) {
        s_tau = T(0);
        s_scal = T(1);
        s_nz = 0;
      } else {
        const T beta = -copysign(sqrt(alpha * alpha + sum), alpha);
        s_tau = (beta - alpha) / beta;
        s_scal = T(1) / (alpha - beta);
        if (own) at(c, jl) = beta;
        s_nz = 1;
      }
    }
    __syncthreads();
    const T tj = s_tau;
    if (s_nz) {
      const T sc = s_scal;
      for (int l = r0 + tid; l < hi; l += NT) at(c, l) *= sc;
    }
    __syncthreads();
    // ---- 2. partial d_t = [own row j] A[j, j0+t] + sum_{own rows i > j} v_i A[i, j0+t]
    T acc[32];
#pragma unroll
    for (int t = 0; t < 32; ++t) acc[t] = T(0);
    for (int l = r0 + tid; l < hi; l += NT) {
      const T vi = at(c, l);
#pragma unroll
      for (int t = 0; t < 32; ++t)
        if (t < jb) acc[t] += vi * P[(int64_t)t * chunk + (l - lo)];
    }
    warp_reduce_scatter32(acc, lane);
    red[warp][lane] = acc[0];
    __syncthreads();
    if (tid < 32) {
      T d = T(0);
#pragma unroll
      for (int w = 0; w < NW; ++w) d += red[w][tid];
      if (own && tid < jb) d += at(tid, jl);
      dot_part[b][tid] = d;
    }
    cluster_sync_all();
    if (tid < 32) {
      T d = T(0);
      for (int r = 0; r < CS; ++r) d += dsmem_load(&dot_part[b][tid], r);
      dvec[tid] = d;
    }
    __syncthreads();
    // ---- 3. apply H_c to the own rows of the remaining columns, extend T
    if (tj != T(0)) {
      for (int t = c + 1; t < jb; ++t) {
        const T f = tj * dvec[t];
        for (int l = r0 + tid; l < hi; l += NT) at(t, l) -= f * at(c, l);
      }
      if (own && tid > c && tid < jb) at(tid, jl) -= tj * dvec[tid];
    }
    if (tid < c) {
      T v = T(0);
      for (int q = tid; q < c; ++q) v += Ts[tid][q] * dvec[q];
      Ts[tid][c] = -tj * v;
    }
    if (tid == 0) {
      Ts[c][c] = tj;
      if (rank == 0) tau[j0 + c] = tj;
    }
    __syncthreads();
  }
  // write back the own rows of the factored panel and of the explicit reflectors
  for (int t = 0; t < jb; ++t) {
    const int jc = j0 + t;
    T* dstA = A + (int64_t)jc * lda + j0;
    T* dst = Vb + (int64_t)jc * ldv + j0;
    for (int l = lo + tid; l < hi; l += NT) {
      const T v = at(t, l);
      dstA[l] = v;
      dst[l] = (l < t) ? T(0) : (l == t ? T(1) : v);
    }
  }
  if (rank == 0)
    for (int e = tid; e < jb * jb; e += NT) {
      const int r = e % jb, cc = e / jb;
      Tm[r + (int64_t)cc * ldt] = Ts[r][cc];
    }
  cluster_sync_all();  // no CTA leaves while another may still read its shared memory
}

// W2[:, c] = op(T) (V^T A[:, c]) for one column c per CTA, jb <= 32:
// the small-M half of applying the block reflector I - V T V^T (op(T) = T^T when
// building R, T when building Q).  V (mr x jb) and A (mr x nc) are column-major.
template <typename T, int NT>
__device__ __forceinline__ void reflector_w_body(const T* __restrict__ V, int ldv, const T* __restrict__ A,
                                                 int lda, int mr, int jb, const T* __restrict__ Tm, int ldt,
                                                 bool transpose_t, T* __restrict__ W2, int c) {
  constexpr int NW = NT / 32;
  __shared__ T red[NW][33];
  __shared__ T w[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const T* a = A + (int64_t)c * lda;
  T acc[32];
#pragma unroll
  for (int t = 0; t < 32; ++t) acc[t] = T(0);
  for (int i = tid; i < mr; i += NT) {
    const T ai = a[i];
#pragma unroll
    for (int t = 0; t < 32; ++t)
      if (t < jb) acc[t] += V[i + (int64_t)t * ldv] * ai;
  }
  warp_reduce_scatter32(acc, lane);
  red[warp][lane] = acc[0];
  __syncthreads();
  if (tid < 32) {
    T v = T(0);
#pragma unroll
    for (int q = 0; q < NW; ++q) v += red[q][tid];
    w[tid] = v;
  }
  __syncthreads();
  if (tid < jb) {
    T v = T(0);
    if (transpose_t) {  // (T^T w)_t = sum_{q <= t} T[q, t] w_q
      for (int q = 0; q <= tid; ++q) v += Tm[q + (int64_t)tid * ldt] * w[q];
    } else {  // (T w)_t = sum_{q >= t} T[t, q] w_q
      for (int q = tid; q < jb; ++q) v += Tm[tid + (int64_t)q * ldt] * w[q];
    }
    W2[tid + (int64_t)c * jb] = v;
  }
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT) reflector_w_kernel(const T* __restrict__ V, int ldv,
                                                         const T* __restrict__ A, int lda, int mr,
                                                         int jb, const T* __restrict__ Tm, int ldt,
                                                         bool transpose_t, T* __restrict__ W2) {
  reflector_w_body<T, NT>(V, ldv, A, lda, mr, jb, Tm, ldt, transpose_t, W2, blockIdx.x);
}

// Batched W2 of the panel at j0 (blockIdx.y = job, blockIdx.x = column): the trailing
// update of the QR (formq = false) or the update of the thin Q being formed.
template <typename T, int NT>
__global__ void __launch_bounds__(NT) reflector_w_batched_kernel(const QrJob<T>* __restrict__ jobs, int j0,
                                                                 int nb, bool formq) {
  const QrJob<T> J = jobs[blockIdx.y];
  const int p = min(J.m, J.n);
  if (j0 >= p) return;
  const int jb = min(nb, p - j0), mr = J.m - j0, c = blockIdx.x;
  const T* V = J.vbuf + j0 + (int64_t)j0 * J.ldv;
  const T* Tm = J.tmat + (int64_t)(j0 / nb) * nb * nb;
  if (!formq) {
    if (c >= J.n - (j0 + jb)) return;
    reflector_w_body<T, NT>(V, J.ldv, J.A + j0 + (int64_t)(j0 + jb) * J.lda, J.lda, mr, jb, Tm, nb, true, J.w2, c);
  } else {
    if (c >= p - j0) return;
    reflector_w_body<T, NT>(V, J.ldv, J.Q + j0 + (int64_t)j0 * J.ldq, J.ldq, mr, jb, Tm, nb, false, J.w2, c);
  }
}

template <typename T>
__global__ void init_thin_q_batched_kernel(const QrJob<T>* __restrict__ jobs) {
  const QrJob<T> J = jobs[blockIdx.y];
  const int p = min(J.m, J.n);
  const int64_t total = (int64_t)J.m * p;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % J.m), c = (int)(e / J.m);
    J.Q[i + (int64_t)c * J.ldq] = (i == c) ? T(1) : T(0);
  }
}

template <typename T>
__global__ void init_thin_q_kernel(T* Q, int m, int p, int ldq) {
  const int64_t total = (int64_t)m * p;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % m), c = (int)(e / m);
    Q[i + (int64_t)c * ldq] = (i == c) ? T(1) : T(0);
  }
}

}  // namespace

constexpr size_t kPanelSmem = 180 * 1024;
constexpr int kClusterSize = 8;       // CTAs sharing one panel
// Panels of at least this many rows go to the cluster kernel; shorter ones stay on one CTA.
template <typename T>
constexpr int cluster_min_rows() {
  return sizeof(T) == 8 ? 256 : 256;
}

template <typename T>
int householder_qr(cudaStream_t s, T* A, int m, int n, int lda, QrWork<T>& w) {
  static int configured[2] = {-1, -1};
  int dev = 0;
  TT_CUDA_CHECK(cudaGetDevice(&dev));
  if (configured[sizeof(T) == 8] != dev) {
    TT_CUDA_CHECK(cudaFuncSetAttribute(qr_panel_kernel<T, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kPanelSmem));
    TT_CUDA_CHECK(cudaFuncSetAttribute(qr_panel_cluster_kernel<T, 256, kClusterSize>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPanelSmem));
    configured[sizeof(T) == 8] = dev;
  }
  const int p = std::min(m, n);
  const int nb = w.nb;
  int panel = 0;
  for (int j0 = 0; j0 < p; j0 += nb, ++panel) {
    const int jb = std::min(nb, p - j0);
    T* Tm = w.tmat + (int64_t)panel * nb * nb;
    const int mr = m - j0;
    const int chunk = (int)ceil_div(mr, kClusterSize);
    const size_t chunk_bytes = (size_t)chunk * jb * sizeof(T);
    if (mr >= cluster_min_rows<T>() && chunk_bytes <= kPanelSmem) {
      // cluster panel: kClusterSize CTAs share the rows
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(kClusterSize);
      cfg.blockDim = dim3(256);
      cfg.dynamicSmemBytes = chunk_bytes;
      cfg.stream = s;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = kClusterSize;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      T* tau = w.tau;
      T* vb = w.vbuf;
      TT_CUDA_CHECK(cudaLaunchKernelEx(&cfg, qr_panel_cluster_kernel<T, 256, kClusterSize>, A, lda, m, j0,
                                       jb, tau, Tm, nb, vb, w.ldv, chunk));
      note_launch();
    } else {
      const size_t panel_bytes = (size_t)mr * jb * sizeof(T);
      const bool staged = panel_bytes <= kPanelSmem;
      qr_panel_kernel<T, 512><<<1, 512, staged ? panel_bytes : 0, s>>>(A, lda, m, j0, jb, w.tau, Tm, nb,
                                                                       w.vbuf, w.ldv, staged);
      TT_LAUNCH_CHECK();
    }
    const int nt = n - (j0 + jb);
    if (nt <= 0) continue;
    const T* V = w.vbuf + j0 + (int64_t)j0 * w.ldv;
    T* At = A + j0 + (int64_t)(j0 + jb) * lda;
    // W2 = T^T (V^T At)   (jb x nt, column-major ld jb)
    reflector_w_kernel<T, 256><<<nt, 256, 0, s>>>(V, w.ldv, At, lda, mr, jb, Tm, nb, true, w.w2);
    TT_LAUNCH_CHECK();
    // At -= V W2
    TT_TRY(gemm_fast<T>(s, mr, nt, jb, -1.0, V, 1, w.ldv, w.w2, 1, jb, 1.0, At, 1, lda, w.status));
  }
  w.m = m;
  w.n = n;
  w.npanels = panel;
  return TT_OK;
}

template <typename T>
int form_thin_q(cudaStream_t s, const QrWork<T>& w, T* Q, int ldq) {
  const int m = w.m, p = std::min(w.m, w.n), nb = w.nb;
  {
    const int64_t total = (int64_t)m * p;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(total, 256), 8192));
    init_thin_q_kernel<T><<<blocks, 256, 0, s>>>(Q, m, p, ldq);
    TT_LAUNCH_CHECK();
  }
  for (int panel = w.npanels - 1; panel >= 0; --panel) {
    const int j0 = panel * nb;
    const int jb = std::min(nb, p - j0);
    const int mr = m - j0, nc = p - j0;
    const T* V = w.vbuf + j0 + (int64_t)j0 * w.ldv;
    const T* Tm = w.tmat + (int64_t)panel * nb * nb;
    T* Qs = Q + j0 + (int64_t)j0 * ldq;
    // W2 = T (V^T Qs) ; Qs -= V W2
    reflector_w_kernel<T, 256><<<nc, 256, 0, s>>>(V, w.ldv, Qs, ldq, mr, jb, Tm, nb, false, w.w2);
    TT_LAUNCH_CHECK();
    TT_TRY(gemm_fast<T>(s, mr, nc, jb, -1.0, V, 1, w.ldv, w.w2, 1, jb, 1.0, Qs, 1, ldq, w.status));
  }
  return TT_OK;
}

// The three GEMMs that apply the panel at j0 of every job to its trailing block X
// (mr x nc, column-major, ld ldx):  W1 = V^T X,  W2 = op(T) W1,  X -= V W2.
// W2 = op(T) V^T X is formed as two GEMMs rather than by one CTA per column: a CTA
// per column re-reads the whole mr x jb reflector panel, which for hundreds of jobs at
// once is tens of GB of L2 traffic per panel; the tiled GEMM reads it once per tile.
template <typename T>
struct PanelGemms {
  std::vector<GemmJob<T, T, T>> w1, w2, up;
  int64_t t1 = 0, t2 = 0, t3 = 0;
  int m1 = 0, n1 = 0, m3 = 0;
  TilePlan p1, p2, p3;  // dense tile plans of the three GEMMs
};

template <typename T>
void panel_gemm_jobs(const QrJob<T>& J, int j0, int nb, bool formq, PanelGemms<T>& G) {
  const int p = std::min(J.m, J.n);
  GemmJob<T, T, T> z{};
  if (j0 >= p) {
    G.w1.push_back(z);
    G.w2.push_back(z);
    G.up.push_back(z);
    return;
  }
  const int jb = std::min(nb, p - j0), mr = J.m - j0;
  T* X;
  int ldx, nc;
  if (!formq) {
    X = J.A + j0 + (int64_t)(j0 + jb) * J.lda;
    ldx = J.lda;
    nc = J.n - (j0 + jb);
  } else {
    X = J.Q + j0 + (int64_t)j0 * J.ldq;
    ldx = J.ldq;
    nc = p - j0;
  }
  if (nc <= 0) {
    G.w1.push_back(z);
    G.w2.push_back(z);
    G.up.push_back(z);
    return;
  }
  const T* V = J.vbuf + j0 + (int64_t)j0 * J.ldv;
  const T* Tm = J.tmat + (int64_t)(j0 / nb) * nb * nb;
  // W1 (jb x nc, ld jb) = V^T X
  G.w1.push_back(GemmJob<T, T, T>{V, X, J.w1, J.ldv, 1, 1, ldx, 1, jb, jb, nc, mr, 1.0, 0.0});
  // W2 = T^T W1 (QR of A) or T W1 (building Q); T is upper triangular, zero below
  if (!formq) G.w2.push_back(GemmJob<T, T, T>{Tm, J.w1, J.w2, nb, 1, 1, jb, 1, jb, jb, nc, jb, 1.0, 0.0});
  else G.w2.push_back(GemmJob<T, T, T>{Tm, J.w1, J.w2, 1, nb, 1, jb, 1, jb, jb, nc, jb, 1.0, 0.0});
  // X -= V W2
  G.up.push_back(GemmJob<T, T, T>{V, J.w2, X, 1, J.ldv, 1, jb, 1, ldx, mr, nc, jb, -1.0, 1.0});
  G.t1 += ceil_div(jb, 64) * ceil_div(nc, 64);
  G.t2 += ceil_div(jb, 64) * ceil_div(nc, 64);
  G.t3 += ceil_div(mr, 64) * ceil_div(nc, 64);
  G.m1 = std::max(G.m1, jb);
  G.n1 = std::max(G.n1, nc);
  G.m3 = std::max(G.m3, mr);
}

// FP32: the three GEMMs in the sliced tensor-core form (exact tensor-core sums; plain FP32
// accumulation of the updates took the error of 20..60-site trains at eps = 1e-6 from
// ~2e-6 to 4.6e-6).  FP64: W2 by the
// reflector kernel (one CTA per column), then the update GEMM - measured faster in FP64,
// where the work is bound by the FP64 pipe rather than by L2 traffic.
// d1..d3: the GEMM jobs of every panel ([panel][job]); e1..e3: their tile prefixes
// ([panel][job + 1]).
template <typename T>
int apply_panels(cudaStream_t s, const QrJob<T>* d_jobs, int nj, int nb, bool formq, int pn,
                 const GemmJob<T, T, T>* d1, const GemmJob<T, T, T>* d2, const GemmJob<T, T, T>* d3,
                 const int* e1, const int* e2, const int* e3, const std::vector<PanelGemms<T>>& meta,
                 unsigned* status) {
  const PanelGemms<T>& M = meta[pn];
  if (M.n1 <= 0) return TT_OK;
  const size_t jo = (size_t)pn * nj, po = (size_t)pn * (nj + 1);
  if (sizeof(T) == 4) {
    TT_TRY((gemm_batched_dense<T, T, T>(s, nj, d1 + jo, e1 + po, M.p1, true, status)));
    TT_TRY((gemm_batched_dense<T, T, T>(s, nj, d2 + jo, e2 + po, M.p2, true, status)));
  } else {
    reflector_w_batched_kernel<T, 256><<<dim3((unsigned)M.n1, (unsigned)nj), 256, 0, s>>>(d_jobs, pn * nb, nb,
                                                                                          formq);
    TT_LAUNCH_CHECK();
  }
  TT_TRY((gemm_batched_dense<T, T, T>(s, nj, d3 + jo, e3 + po, M.p3, true, status)));
  return TT_OK;
}

template <typename T>
struct PanelArrays {
  const GemmJob<T, T, T> *d1 = nullptr, *d2 = nullptr, *d3 = nullptr;
  const int *e1 = nullptr, *e2 = nullptr, *e3 = nullptr;
};

template <typename T>
int build_panel_gemms(cudaStream_t s, const std::vector<QrJob<T>>& hj, int nb, bool formq, int npanels,
                      JobArena& arena, std::vector<PanelGemms<T>>& meta, PanelArrays<T>& D) {
  const int nj = (int)hj.size();
  meta.assign(npanels, PanelGemms<T>{});
  std::vector<GemmJob<T, T, T>> a1, a2, a3;
  std::vector<int> q1((size_t)npanels * (nj + 1)), q2(q1.size()), q3(q1.size());
  for (int pn = 0; pn < npanels; ++pn) {
    PanelGemms<T>& M = meta[pn];
    for (const auto& J : hj) panel_gemm_jobs(J, pn * nb, nb, formq, M);
    const size_t po = (size_t)pn * (nj + 1);
    M.p1 = tile_prefix(M.w1.data(), nj, q1.data() + po);
    M.p2 = tile_prefix(M.w2.data(), nj, q2.data() + po);
    M.p3 = tile_prefix(M.up.data(), nj, q3.data() + po);
    a1.insert(a1.end(), M.w1.begin(), M.w1.end());
    a2.insert(a2.end(), M.w2.begin(), M.w2.end());
    a3.insert(a3.end(), M.up.begin(), M.up.end());
  }
  D.d1 = arena.push(a1, s);
  D.d2 = arena.push(a2, s);
  D.d3 = arena.push(a3, s);
  D.e1 = arena.push(q1, s);
  D.e2 = arena.push(q2, s);
  D.e3 = arena.push(q3, s);
  if (!D.d1 || !D.d2 || !D.d3 || !D.e1 || !D.e2 || !D.e3) return fail(TT_ERR_WORKSPACE, "batched QR: job arena full");
  return TT_OK;
}

// FP32 jobs with FP64 scratch: the panel at column j0 of every job copied into its FP64
// scratch (rows j0..m-1 as rows 0..mr-1), factored there by the FP64 panel kernel, and
// R, the reflectors, T and tau written back rounded to FP32.  The FP32 panel's own
// arithmetic (reflectors formed and applied in FP32 inside the panel) left the mixed
// form ~2e-6 from the unrounded trains; with FP64 panels it stays below 1e-6, while the
// trailing updates remain in the FP32 GEMMs (sliced tensor-core form or Dot2).
int panel_f64(cudaStream_t s, const std::vector<QrJob<float>>& hj, int j0, int nb, JobArena& arena) {
  std::vector<MapJob> to64, back;
  std::vector<QrJob<double>> dj;
  int64_t mx = 1;
  int mr_max = 0;
  for (const auto& J : hj) {
    const int p = std::min(J.m, J.n);
    if (j0 >= p) continue;
    const int jb = std::min(nb, p - j0), mr = J.m - j0;
    float* Ablk = J.A + j0 + (int64_t)j0 * J.lda;
    to64.push_back(MapJob{Ablk, J.p64, mr, jb, 1, J.lda, 1, mr, MAP_COPY});
    QrJob<double> D{};
    D.A = J.p64;
    D.m = mr;
    D.n = jb;
    D.lda = mr;
    D.tau = J.tau64;
    D.tmat = J.t64;
    D.vbuf = J.v64;
    D.ldv = mr;
    dj.push_back(D);
    back.push_back(MapJob{J.p64, Ablk, mr, jb, 1, mr, 1, J.lda, MAP_COPY});
    back.push_back(MapJob{J.v64, J.vbuf + j0 + (int64_t)j0 * J.ldv, mr, jb, 1, mr, 1, J.ldv, MAP_COPY});
    back.push_back(MapJob{J.t64, J.tmat + (int64_t)(j0 / nb) * nb * nb, jb, jb, 1, nb, 1, nb, MAP_COPY});
    back.push_back(MapJob{J.tau64, J.tau + j0, jb, 1, 1, jb, 1, jb, MAP_COPY});
    mx = std::max<int64_t>(mx, (int64_t)mr * jb);
    mr_max = std::max(mr_max, mr);
  }
  if (dj.empty()) return TT_OK;
  const MapJob* d_to = arena.push(to64, s);
  const MapJob* d_back = arena.push(back, s);
  const QrJob<double>* d_dj = arena.push(dj, s);
  if (!d_to || !d_back || !d_dj) return fail(TT_ERR_WORKSPACE, "batched QR: job arena full");
  TT_TRY((map_batched<float, double>(s, (int)to64.size(), d_to, mx)));
  const size_t smem = std::min(kPanelSmem, (size_t)mr_max * nb * sizeof(double));
  qr_panel_batched_kernel<double, 512><<<(unsigned)dj.size(), 512, smem, s>>>(d_dj, 0, nb, smem);
  TT_LAUNCH_CHECK();
  return map_batched<double, float>(s, (int)back.size(), d_back, mx);
}

template <typename T>
int householder_qr_batched(cudaStream_t s, const std::vector<QrJob<T>>& hj, const QrJob<T>* d_jobs, int nb,
                           JobArena& arena, unsigned* status) {
  const int nj = (int)hj.size();
  if (nj == 0) return TT_OK;
  if (nj > 65535) return fail(TT_ERR_UNSUPPORTED, "householder_qr_batched: too many jobs");
  static int configured[2] = {-1, -1};
  int dev = 0;
  TT_CUDA_CHECK(cudaGetDevice(&dev));
  if (configured[sizeof(T) == 8] != dev) {
    TT_CUDA_CHECK(cudaFuncSetAttribute(qr_panel_batched_kernel<T, 512>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPanelSmem));
    TT_CUDA_CHECK(cudaFuncSetAttribute(qr_panel_batched_kernel<double, 512>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPanelSmem));
    configured[sizeof(T) == 8] = dev;
  }
  bool f64_panels = false;
  if constexpr (std::is_same<T, float>::value) f64_panels = hj[0].p64 != nullptr;
  int p_max = 0, m_max = 0;
  for (const auto& J : hj) {
    p_max = std::max(p_max, std::min(J.m, J.n));
    m_max = std::max(m_max, J.m);
  }
  const int npanels = (int)ceil_div(p_max, nb);
  std::vector<PanelGemms<T>> meta;
  PanelArrays<T> D;
  TT_TRY(build_panel_gemms(s, hj, nb, false, npanels, arena, meta, D));
  for (int pn = 0; pn < npanels; ++pn) {
    const int j0 = pn * nb;
    if constexpr (std::is_same<T, float>::value) {
      if (f64_panels) {
        TT_TRY(panel_f64(s, hj, j0, nb, arena));
        TT_TRY(apply_panels(s, d_jobs, nj, nb, false, pn, D.d1, D.d2, D.d3, D.e1, D.e2, D.e3, meta, status));
        continue;
      }
    }
    const size_t smem = std::min(kPanelSmem, (size_t)(m_max - j0) * nb * sizeof(T));
    qr_panel_batched_kernel<T, 512><<<nj, 512, smem, s>>>(d_jobs, j0, nb, smem);
    TT_LAUNCH_CHECK();
    TT_TRY(apply_panels(s, d_jobs, nj, nb, false, pn, D.d1, D.d2, D.d3, D.e1, D.e2, D.e3, meta, status));
  }
  return TT_OK;
}

template <typename T>
int form_thin_q_batched(cudaStream_t s, const std::vector<QrJob<T>>& hj, const QrJob<T>* d_jobs, int nb,
                        JobArena& arena, unsigned* status) {
  const int nj = (int)hj.size();
  if (nj == 0) return TT_OK;
  int p_max = 0;
  int64_t qmax = 1;
  for (const auto& J : hj) {
    const int p = std::min(J.m, J.n);
    p_max = std::max(p_max, p);
    qmax = std::max<int64_t>(qmax, (int64_t)J.m * p);
  }
  init_thin_q_batched_kernel<T><<<dim3((unsigned)std::min<int64_t>(ceil_div(qmax, 256), 1024), (unsigned)nj), 256,
                                  0, s>>>(d_jobs);
  TT_LAUNCH_CHECK();
  const int npanels = (int)ceil_div(p_max, nb);
  std::vector<PanelGemms<T>> meta;
  PanelArrays<T> D;
  TT_TRY(build_panel_gemms(s, hj, nb, true, npanels, arena, meta, D));
  for (int pn = npanels - 1; pn >= 0; --pn)
    TT_TRY(apply_panels(s, d_jobs, nj, nb, true, pn, D.d1, D.d2, D.d3, D.e1, D.e2, D.e3, meta, status));
  return TT_OK;
}

template int householder_qr_batched<double>(cudaStream_t, const std::vector<QrJob<double>>&, const QrJob<double>*,
                                            int, JobArena&, unsigned*);
template int householder_qr_batched<float>(cudaStream_t, const std::vector<QrJob<float>>&, const QrJob<float>*,
                                           int, JobArena&, unsigned*);
template int form_thin_q_batched<double>(cudaStream_t, const std::vector<QrJob<double>>&, const QrJob<double>*,
                                         int, JobArena&, unsigned*);
template int form_thin_q_batched<float>(cudaStream_t, const std::vector<QrJob<float>>&, const QrJob<float>*,
                                        int, JobArena&, unsigned*);
template int householder_qr<double>(cudaStream_t, double*, int, int, int, QrWork<double>&);
template int householder_qr<float>(cudaStream_t, float*, int, int, int, QrWork<float>&);
template int form_thin_q<double>(cudaStream_t, const QrWork<double>&, double*, int);
template int form_thin_q<float>(cudaStream_t, const QrWork<float>&, float*, int);

}  // namespace tt
