// Strided SIMT GEMM with FP64 accumulation:  C = alpha * A B + beta * C.
// A is M x K with element (m, k) at A[m*sam + k*sak], B is K x N with (k, n) at
// B[k*sbk + n*sbn], C is M x N with (m, n) at C[m*scm + n*scn].  Any of the
// operands may be row- or column-major (or a strided slice of a core), so the
// rounding sweeps and the environment sweeps need no explicit transposes.
//
// This is the GEMM of the plain FP64 form (DFMA-bound on GB300: ~1.2 TFLOP/s peak)
// and of the FP64 environment sweeps.  64 x 64 x 16 tiles, 256 threads, 4 x 4
// outputs per thread, tiles staged in shared memory.
#include <type_traits>

#include "tt_gemm.cuh"

namespace tt {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

template <typename TA, typename TB, typename TC>
__global__ void __launch_bounds__(NT) gemm_simt_kernel(int M, int N, int K, double alpha,
                                                       const TA* __restrict__ A, int64_t sam,
                                                       int64_t sak, const TB* __restrict__ B,
                                                       int64_t sbk, int64_t sbn, double beta,
                                                       TC* __restrict__ C, int64_t scm,
                                                       int64_t scn) {
  // FP32 operands and output accumulate in FP32 (mixed form), anything else in FP64
  using Acc = std::conditional_t<std::is_same<TA, float>::value && std::is_same<TB, float>::value &&
                                     std::is_same<TC, float>::value,
                                 float, double>;
  __shared__ Acc As[BK][BM + 1];
  __shared__ Acc Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  Acc acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = Acc(0);

  const bool a_m_fast = (sam == 1);
  const bool b_n_fast = (sbn == 1);

  for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
    for (int u = 0; u < (BM * BK) / NT; ++u) {
      const int e = tid + u * NT;
      int mm, kk;
      if (a_m_fast) {
        mm = e % BM;
        kk = e / BM;
      } else {
        kk = e % BK;
        mm = e / BK;
      }
      const int gm = m0 + mm, gk = k0 + kk;
      Acc v = Acc(0);
      if (gm < M && gk < K) v = (Acc)A[(int64_t)gm * sam + (int64_t)gk * sak];
      As[kk][mm] = v;
    }
#pragma unroll
    for (int u = 0; u < (BN * BK) / NT; ++u) {
      const int e = tid + u * NT;
      int nn, kk;
      if (b_n_fast) {
        nn = e % BN;
        kk = e / BN;
      } else {
        kk = e % BK;
        nn = e / BK;
      }
      const int gn = n0 + nn, gk = k0 + kk;
      Acc v = Acc(0);
      if (gn < N && gk < K) v = (Acc)B[(int64_t)gk * sbk + (int64_t)gn * sbn];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      Acc a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx + 16 * j;
      if (gn >= N) continue;
      TC* p = C + (int64_t)gm * scm + (int64_t)gn * scn;
      double v = alpha * (double)acc[i][j];
      if (beta != 0.0) v += beta * (double)(*p);
      *p = (TC)v;
    }
  }
}

template <typename TC>
__global__ void scale_kernel(int M, int N, double beta, TC* C, int64_t scm, int64_t scn) {
  const int64_t total = (int64_t)M * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int m = (int)(e / N), n = (int)(e % N);
    TC* p = C + (int64_t)m * scm + (int64_t)n * scn;
    *p = (beta == 0.0) ? TC(0) : (TC)(beta * (double)(*p));
  }
}

}  // namespace

template <typename TA, typename TB, typename TC>
int gemm(cudaStream_t s, int M, int N, int K, double alpha, const TA* A, int64_t sam, int64_t sak,
         const TB* B, int64_t sbk, int64_t sbn, double beta, TC* C, int64_t scm, int64_t scn) {
  if (M <= 0 || N <= 0) return TT_OK;
  if (K <= 0) {
    if (beta == 1.0) return TT_OK;
    const int64_t total = (int64_t)M * N;
    const int blocks = (int)std::min<int64_t>(ceil_div(total, 256), 4096);
    scale_kernel<TC><<<blocks, 256, 0, s>>>(M, N, beta, C, scm, scn);
    TT_LAUNCH_CHECK();
    return TT_OK;
  }
  dim3 grid((unsigned)ceil_div(N, BN), (unsigned)ceil_div(M, BM));
  if (grid.y > 65535u) return fail(TT_ERR_UNSUPPORTED, "gemm: M too large");
  gemm_simt_kernel<TA, TB, TC>
      <<<grid, NT, 0, s>>>(M, N, K, alpha, A, sam, sak, B, sbk, sbn, beta, C, scm, scn);
  TT_LAUNCH_CHECK();
  return TT_OK;
}

#define TT_GEMM_INST(TA, TB, TC)                                                           \
  template int gemm<TA, TB, TC>(cudaStream_t, int, int, int, double, const TA*, int64_t, \
                                int64_t, const TB*, int64_t, int64_t, double, TC*, int64_t, \
                                int64_t);
TT_GEMM_INST(double, double, double)
TT_GEMM_INST(double, double, float)
TT_GEMM_INST(double, float, double)
TT_GEMM_INST(double, float, float)
TT_GEMM_INST(float, double, double)
TT_GEMM_INST(float, double, float)
TT_GEMM_INST(float, float, double)
TT_GEMM_INST(float, float, float)
#undef TT_GEMM_INST

template <>
int gemm_fast<double>(cudaStream_t s, int M, int N, int K, double alpha, const double* A, int64_t sam,
                      int64_t sak, const double* B, int64_t sbk, int64_t sbn, double beta, double* C,
                      int64_t scm, int64_t scn, unsigned* status) {
  (void)status;
  return gemm<double, double, double>(s, M, N, K, alpha, A, sam, sak, B, sbk, sbn, beta, C, scm, scn);
}

template <>
int gemm_fast<float>(cudaStream_t s, int M, int N, int K, double alpha, const float* A, int64_t sam,
                     int64_t sak, const float* B, int64_t sbk, int64_t sbn, double beta, float* C,
                     int64_t scm, int64_t scn, unsigned* status) {
  // tiny products stay on the SIMT path (a 128-row tensor-core tile would be mostly padding)
  if ((int64_t)M * N * K < (1 << 16) || K < 8)
    return gemm<float, float, float>(s, M, N, K, alpha, A, sam, sak, B, sbk, sbn, beta, C, scm, scn);
  return gemm_tf32x3(s, M, N, K, alpha, A, sam, sak, B, sbk, sbn, beta, C, scm, scn, status);
}

}  // namespace tt
