// Strided SIMT GEMM with FP64 accumulation:  C = alpha * A B + beta * C.
// A is M x K with element (m, k) at A[m*sam + k*sak], B is K x N with (k, n) at
// B[k*sbk + n*sbn], C is M x N with (m, n) at C[m*scm + n*scn].  Any of the
// operands may be row- or column-major (or a strided slice of a core), so the
// rounding sweeps and the environment sweeps need no explicit transposes.
//
// This is the GEMM of the plain FP64 form (DFMA-bound on GB300: ~1.2 TFLOP/s peak)
// and of the FP64 environment sweeps.  64 x 64 x 16 tiles, 256 threads, 4 x 4
// outputs per thread, tiles staged in shared memory.
//
// When all three operands are FP32 (the mixed form) the dot products are compensated
// instead (Ogita, Rump & Oishi 2005, "Accurate sum and dot product", Dot2): each
// product is split exactly as p + e with one FMA (TwoProduct), the running sum s
// takes p through an error-free TwoSum, and the rounding errors are collected in a
// second FP32 accumulator.  The result is as accurate as if computed in about twice
// the working precision and then rounded, at ~10 FP32 operations per multiply-add:
// several times the throughput of FP64 arithmetic on GB300, whose FP64 rate is about
// one sixtieth of its FP32 rate.  FP32 products large enough to give every SM a
// 128 x 64 tile go to the sliced tensor-core form instead (tt_gemm_tc.cu), which is as
// accurate for these uses and several times faster.
#include <type_traits>

#include "tt_gemm.cuh"

namespace tt {

namespace {

constexpr int BK = 16, NT = 256;

// BM x BN tile (bx, by) of C, 16 x 16 threads, (BM / 16) x (BN / 16) outputs per thread.
// COMP: compensated (Dot2) accumulation when all operands are FP32.
template <int BM, int BN, typename TA, typename TB, typename TC, bool COMP = true>
__device__ __forceinline__ void gemm_tile(int M, int N, int K, double alpha, const TA* __restrict__ A,
                                          int64_t sam, int64_t sak, const TB* __restrict__ B, int64_t sbk,
                                          int64_t sbn, double beta, TC* __restrict__ C, int64_t scm,
                                          int64_t scn, int bx, int by) {
  // FP32 A and B: compensated FP32 (Dot2) into an FP32 or FP64 C (plain FP32 sums if !COMP
  // and C is FP32).  FP32 A, FP64 B, FP32 C (the mixed form's update X -= V W2 with W2 in
  // FP64): Dot2 with B split into hi + lo FP32 words, a b = a b_hi (exact TwoProduct) +
  // a b_lo.  Every other combination in FP64.
  constexpr bool kF32AB = std::is_same<TA, float>::value && std::is_same<TB, float>::value;
  constexpr bool kAllF32 = kF32AB && std::is_same<TC, float>::value;
  constexpr bool kSplitB = COMP && std::is_same<TA, float>::value && std::is_same<TB, double>::value &&
                           std::is_same<TC, float>::value;
  constexpr bool kDot2 = COMP && (kF32AB || kSplitB);
  using Acc = std::conditional_t<(kAllF32 || kDot2), float, double>;
  __shared__ Acc As[BK][BM + 1];
  __shared__ Acc Bs[BK][BN + 1];
  __shared__ Acc Bl[kSplitB ? BK : 1][kSplitB ? BN + 1 : 1];  // low words of B (kSplitB)
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = by * BM, n0 = bx * BN;
  constexpr int TM = BM / 16, TN = BN / 16;
  Acc acc[TM][TN], cmp[TM][TN];  // cmp: the collected rounding errors (Dot2 only)
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = cmp[i][j] = Acc(0);

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
      if constexpr (kSplitB) {
        double v = 0.0;
        if (gn < N && gk < K) v = (double)B[(int64_t)gk * sbk + (int64_t)gn * sbn];
        const float h = (float)v;
        Bs[kk][nn] = h;
        Bl[kk][nn] = (float)(v - (double)h);
      } else {
        Acc v = Acc(0);
        if (gn < N && gk < K) v = (Acc)B[(int64_t)gk * sbk + (int64_t)gn * sbn];
        Bs[kk][nn] = v;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      Acc a[TM], b[TN], bl[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        b[j] = Bs[kk][tx + 16 * j];
        if constexpr (kSplitB) bl[j] = Bl[kk][tx + 16 * j];
        else bl[j] = Acc(0);
      }
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          if constexpr (kDot2) {
            const float p = __fmul_rn(a[i], b[j]);
            float e = __fmaf_rn(a[i], b[j], -p);  // a b = p + e exactly
            if constexpr (kSplitB) e = __fmaf_rn(a[i], bl[j], e);
            const float x = acc[i][j];
            const float t = __fadd_rn(x, p);  // TwoSum: x + p = t + f exactly
            const float z = __fsub_rn(t, x);
            const float f = __fadd_rn(__fsub_rn(x, __fsub_rn(t, z)), __fsub_rn(p, z));
            acc[i][j] = t;
            cmp[i][j] = __fadd_rn(cmp[i][j], __fadd_rn(f, e));
          } else {
            acc[i][j] = fma(a[i], b[j], acc[i][j]);
          }
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gn = n0 + tx + 16 * j;
      if (gn >= N) continue;
      TC* p = C + (int64_t)gm * scm + (int64_t)gn * scn;
      double v = alpha * ((double)acc[i][j] + (double)cmp[i][j]);
      if (beta != 0.0) v += beta * (double)(*p);
      *p = (TC)v;
    }
  }
}

template <int BM, int BN, typename TA, typename TB, typename TC, bool COMP>
__global__ void __launch_bounds__(NT) gemm_simt_kernel(int M, int N, int K, double alpha,
                                                       const TA* __restrict__ A, int64_t sam,
                                                       int64_t sak, const TB* __restrict__ B,
                                                       int64_t sbk, int64_t sbn, double beta,
                                                       TC* __restrict__ C, int64_t scm,
                                                       int64_t scn) {
  gemm_tile<BM, BN, TA, TB, TC, COMP>(M, N, K, alpha, A, sam, sak, B, sbk, sbn, beta, C, scm, scn, blockIdx.x,
                                      blockIdx.y);
}

// One GEMM per blockIdx.z; tiles outside a job's M x N exit at once.
template <int BM, int BN, typename TA, typename TB, typename TC, bool COMP>
__global__ void __launch_bounds__(NT) gemm_batched_kernel(const GemmJob<TA, TB, TC>* __restrict__ jobs) {
  const GemmJob<TA, TB, TC> j = jobs[blockIdx.z];
  if ((int)blockIdx.y * BM >= j.M || (int)blockIdx.x * BN >= j.N || j.K <= 0) return;
  gemm_tile<BM, BN, TA, TB, TC, COMP>(j.M, j.N, j.K, j.alpha, j.A, j.sam, j.sak, j.B, j.sbk, j.sbn, j.beta, j.C,
                                      j.scm, j.scn, blockIdx.x, blockIdx.y);
}

// Dense batched form: one CTA per real tile.  prefix[j] = tiles of jobs 0..j-1 (njobs + 1
// entries); a CTA finds its job by binary search and its tile from the remainder, so no
// CTA is spent on the empty tiles of a grid sized for the largest job.
template <int BM, int BN, typename TA, typename TB, typename TC, bool COMP>
__global__ void __launch_bounds__(NT) gemm_dense_kernel(const GemmJob<TA, TB, TC>* __restrict__ jobs,
                                                        const int* __restrict__ prefix, int njobs) {
  const int id = blockIdx.x;
  int lo = 0, hi = njobs;  // last job with prefix[job] <= id
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (prefix[mid] <= id) lo = mid;
    else hi = mid;
  }
  const GemmJob<TA, TB, TC> j = jobs[lo];
  const int local = id - prefix[lo];
  const int tn = (j.N + BN - 1) / BN;
  gemm_tile<BM, BN, TA, TB, TC, COMP>(j.M, j.N, j.K, j.alpha, j.A, j.sam, j.sak, j.B, j.sbk, j.sbn, j.beta, j.C,
                                      j.scm, j.scn, local % tn, local / tn);
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

template <typename TA, typename TB, typename TC, bool COMP>
int gemm_launch(cudaStream_t s, int M, int N, int K, double alpha, const TA* A, int64_t sam, int64_t sak,
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
  // 64 x 64 tiles while they give at least one CTA per SM; 32 x 32 tiles below that, so
  // that small products (the rank-nb updates of the QR, K = nb) still spread over the
  // SMs: a 64 x 64 x 16 FP64 tile is ~16 us of one SM's 2 DFMA / clock.
  const int64_t big = ceil_div(N, 64) * ceil_div(M, 64);
  if (big >= num_sms()) {
    dim3 grid((unsigned)ceil_div(N, 64), (unsigned)ceil_div(M, 64));
    if (grid.y > 65535u) return fail(TT_ERR_UNSUPPORTED, "gemm: M too large");
    gemm_simt_kernel<64, 64, TA, TB, TC, COMP>
        <<<grid, NT, 0, s>>>(M, N, K, alpha, A, sam, sak, B, sbk, sbn, beta, C, scm, scn);
  } else {
    dim3 grid((unsigned)ceil_div(N, 32), (unsigned)ceil_div(M, 32));
    if (grid.y > 65535u) return fail(TT_ERR_UNSUPPORTED, "gemm: M too large");
    gemm_simt_kernel<32, 32, TA, TB, TC, COMP>
        <<<grid, NT, 0, s>>>(M, N, K, alpha, A, sam, sak, B, sbk, sbn, beta, C, scm, scn);
  }
  TT_LAUNCH_CHECK();
  return TT_OK;
}

template <typename TA, typename TB, typename TC>
int gemm(cudaStream_t s, int M, int N, int K, double alpha, const TA* A, int64_t sam, int64_t sak,
         const TB* B, int64_t sbk, int64_t sbn, double beta, TC* C, int64_t scm, int64_t scn) {
  return gemm_launch<TA, TB, TC, true>(s, M, N, K, alpha, A, sam, sak, B, sbk, sbn, beta, C, scm, scn);
}

template <typename TA, typename TB, typename TC>
int gemm_batched(cudaStream_t s, int njobs, const GemmJob<TA, TB, TC>* d_jobs, int M_max, int N_max,
                 int64_t tiles64, bool compensated) {
  if (njobs <= 0 || M_max <= 0 || N_max <= 0) return TT_OK;
  if (njobs > 65535) return fail(TT_ERR_UNSUPPORTED, "gemm_batched: too many jobs");
  if (tiles64 >= num_sms()) {
    dim3 grid((unsigned)ceil_div(N_max, 64), (unsigned)ceil_div(M_max, 64), (unsigned)njobs);
    if (grid.y > 65535u) return fail(TT_ERR_UNSUPPORTED, "gemm_batched: M too large");
    if (compensated) gemm_batched_kernel<64, 64, TA, TB, TC, true><<<grid, NT, 0, s>>>(d_jobs);
    else gemm_batched_kernel<64, 64, TA, TB, TC, false><<<grid, NT, 0, s>>>(d_jobs);
  } else {
    dim3 grid((unsigned)ceil_div(N_max, 32), (unsigned)ceil_div(M_max, 32), (unsigned)njobs);
    if (grid.y > 65535u) return fail(TT_ERR_UNSUPPORTED, "gemm_batched: M too large");
    if (compensated) gemm_batched_kernel<32, 32, TA, TB, TC, true><<<grid, NT, 0, s>>>(d_jobs);
    else gemm_batched_kernel<32, 32, TA, TB, TC, false><<<grid, NT, 0, s>>>(d_jobs);
  }
  TT_LAUNCH_CHECK();
  return TT_OK;
}

template <typename TA, typename TB, typename TC>
TilePlan tile_prefix(const GemmJob<TA, TB, TC>* jobs, int njobs, int* prefix) {
  TilePlan plan;
  if constexpr (std::is_same_v<TA, float> && std::is_same_v<TB, float> && std::is_same_v<TC, float>) {
    // the sliced tensor-core form when its 128 x 64 tiles give every SM a CTA; below that
    // the SIMT tiles, up to 8x more CTAs, finish first
    int64_t sl = 0;
    for (int i = 0; i < njobs; ++i) {
      if (jobs[i].K > 0) sl += sliced_tiles(jobs[i].M, jobs[i].N);
      plan.K_max = std::max(plan.K_max, jobs[i].K);
    }
    if (sl >= num_sms()) {
      plan.tile = kSlicedPlan;
      int64_t acc = 0;
      for (int i = 0; i < njobs; ++i) {
        prefix[i] = (int)acc;
        if (jobs[i].K > 0) acc += sliced_tiles(jobs[i].M, jobs[i].N);
      }
      prefix[njobs] = (int)acc;
      plan.total = acc;
      return plan;
    }
  }
  int64_t t64 = 0;
  for (int i = 0; i < njobs; ++i)
    if (jobs[i].M > 0 && jobs[i].N > 0 && jobs[i].K > 0) t64 += ceil_div(jobs[i].M, 64) * ceil_div(jobs[i].N, 64);
  plan.tile = t64 >= num_sms() ? 64 : 32;
  int64_t acc = 0;
  for (int i = 0; i < njobs; ++i) {
    prefix[i] = (int)acc;
    if (jobs[i].M > 0 && jobs[i].N > 0 && jobs[i].K > 0)
      acc += ceil_div(jobs[i].M, plan.tile) * ceil_div(jobs[i].N, plan.tile);
  }
  prefix[njobs] = (int)acc;
  plan.total = acc;
  return plan;
}

template <typename TA, typename TB, typename TC>
int gemm_batched_dense(cudaStream_t s, int njobs, const GemmJob<TA, TB, TC>* d_jobs, const int* d_prefix,
                       const TilePlan& plan, bool compensated, unsigned* status) {
  if (njobs <= 0 || plan.total <= 0) return TT_OK;
  if constexpr (std::is_same_v<TA, float> && std::is_same_v<TB, float> && std::is_same_v<TC, float>) {
    if (plan.tile == kSlicedPlan) return gemm_sliced_dense(s, njobs, d_jobs, d_prefix, plan.total, plan.K_max, status);
  }
  if (plan.total > 0x7fffffff) return fail(TT_ERR_UNSUPPORTED, "gemm_batched_dense: too many tiles");
  const unsigned g = (unsigned)plan.total;
  if (plan.tile == 64) {
    if (compensated) gemm_dense_kernel<64, 64, TA, TB, TC, true><<<g, NT, 0, s>>>(d_jobs, d_prefix, njobs);
    else gemm_dense_kernel<64, 64, TA, TB, TC, false><<<g, NT, 0, s>>>(d_jobs, d_prefix, njobs);
  } else {
    if (compensated) gemm_dense_kernel<32, 32, TA, TB, TC, true><<<g, NT, 0, s>>>(d_jobs, d_prefix, njobs);
    else gemm_dense_kernel<32, 32, TA, TB, TC, false><<<g, NT, 0, s>>>(d_jobs, d_prefix, njobs);
  }
  TT_LAUNCH_CHECK();
  return TT_OK;
}

#define TT_GEMM_INST(TA, TB, TC)                                                           \
  template int gemm<TA, TB, TC>(cudaStream_t, int, int, int, double, const TA*, int64_t, \
                                int64_t, const TB*, int64_t, int64_t, double, TC*, int64_t, \
                                int64_t);                                                  \
  template int gemm_batched<TA, TB, TC>(cudaStream_t, int, const GemmJob<TA, TB, TC>*, int, int, int64_t, bool); \
  template TilePlan tile_prefix<TA, TB, TC>(const GemmJob<TA, TB, TC>*, int, int*);                            \
  template int gemm_batched_dense<TA, TB, TC>(cudaStream_t, int, const GemmJob<TA, TB, TC>*, const int*,       \
                                              const TilePlan&, bool, unsigned*);
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
int gemm_core<double>(cudaStream_t s, int M, int N, int K, double alpha, const double* A, int64_t sam,
                      int64_t sak, const double* B, int64_t sbk, int64_t sbn, double beta, double* C,
                      int64_t scm, int64_t scn, unsigned* status) {
  (void)status;
  return gemm<double, double, double>(s, M, N, K, alpha, A, sam, sak, B, sbk, sbn, beta, C, scm, scn);
}

template <>
int gemm_core<float>(cudaStream_t s, int M, int N, int K, double alpha, const float* A, int64_t sam,
                     int64_t sak, const float* B, int64_t sbk, int64_t sbn, double beta, float* C,
                     int64_t scm, int64_t scn, unsigned* status) {
  if (K >= 16 && sliced_tiles(M, N) >= num_sms())
    return gemm_sliced(s, M, N, K, alpha, A, sam, sak, B, sbk, sbn, beta, C, scm, scn, status);
  return gemm<float, float, float>(s, M, N, K, alpha, A, sam, sak, B, sbk, sbn, beta, C, scm, scn);
}

template <>
int gemm_fast<float>(cudaStream_t s, int M, int N, int K, double alpha, const float* A, int64_t sam,
                     int64_t sak, const float* B, int64_t sbk, int64_t sbn, double beta, float* C,
                     int64_t scm, int64_t scn, unsigned* status) {
  return gemm_core<float>(s, M, N, K, alpha, A, sam, sak, B, sbk, sbn, beta, C, scm, scn, status);
}

}  // namespace tt
