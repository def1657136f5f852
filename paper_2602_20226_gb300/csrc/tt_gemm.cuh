// GEMM entry points used inside libtt.
#pragma once

#include <algorithm>

#include "tt_common.cuh"

namespace tt {

// C = alpha * A B + beta * C with arbitrary element strides (see tt_gemm.cu).
// Compensated FP32 dot products (Dot2) when every operand is FP32, FP64 otherwise;
// beta == 0 never reads C.
template <typename TA, typename TB, typename TC>
int gemm(cudaStream_t s, int M, int N, int K, double alpha, const TA* A, int64_t sam, int64_t sak,
         const TB* B, int64_t sbk, int64_t sbn, double beta, TC* C, int64_t scm, int64_t scn);

// One C = alpha A B + beta C of a batch (strides as in gemm); beta == 0 never reads C.
template <typename TA, typename TB, typename TC>
struct GemmJob {
  const TA* A;
  const TB* B;
  TC* C;
  int64_t sam, sak, sbk, sbn, scm, scn;
  int M, N, K;
  double alpha, beta;
};

// All jobs of d_jobs (device array) in one launch; M_max / N_max bound every job's M / N,
// tiles64 = sum over jobs of their 64 x 64 tile counts (picks the tile size).
// compensated: Dot2 accumulation when all operands are FP32 (plain FP32 FMA otherwise).
template <typename TA, typename TB, typename TC>
int gemm_batched(cudaStream_t s, int njobs, const GemmJob<TA, TB, TC>* d_jobs, int M_max, int N_max,
                 int64_t tiles64, bool compensated = true);

// Dense batched form: prefix (njobs + 1 host ints) = running tile counts for the tile size
// the plan picks (all-FP32 jobs: the sliced tensor-core form, plan.tile == kSlicedPlan,
// when its tiles give every SM a CTA; otherwise 64 x 64 SIMT tiles when they do, else
// 32 x 32); the same array in device memory goes to gemm_batched_dense, which launches
// one CTA per real tile.
struct TilePlan {
  int tile = 64;
  int64_t total = 0;
  int K_max = 0;  // largest K of the jobs
};
template <typename TA, typename TB, typename TC>
TilePlan tile_prefix(const GemmJob<TA, TB, TC>* jobs, int njobs, int* prefix);
template <typename TA, typename TB, typename TC>
int gemm_batched_dense(cudaStream_t s, int njobs, const GemmJob<TA, TB, TC>* d_jobs, const int* d_prefix,
                       const TilePlan& plan, bool compensated = true, unsigned* status = nullptr);

// FP32 GEMM on the tensor cores in the sliced form (tt_gemm_tc.cu): per 32-wide K block
// each row of A and column of B is scaled by its own power of two and cut into three
// balanced integer slices; the tensor cores sum the slice products exactly (integers
// below 2^24) and the block sums are added in float-float.  Error <= ~2^-25 sum_k
// max|a| max|b| per element (maxima over the K block), zero-mean.  status: ST_TIMEOUT if
// an mbarrier wait expired (may be null).
int gemm_sliced(cudaStream_t s, int M, int N, int K, double alpha, const float* A, int64_t sam, int64_t sak,
                const float* B, int64_t sbk, int64_t sbn, double beta, float* C, int64_t scm, int64_t scn,
                unsigned* status);
// tiles of one job in the sliced form (128 x 64, the short side first when M is short)
int64_t sliced_tiles(int M, int N);
// dense batched sliced form: prefix from tile_prefix with plan.tile == kSlicedPlan;
// K_max >= every job's K (K_max <= 32: the one-block kernel, two CTAs per SM)
int gemm_sliced_dense(cudaStream_t s, int njobs, const GemmJob<float, float, float>* d_jobs, const int* d_prefix,
                      int64_t total_tiles, int K_max, unsigned* status);
constexpr int kSlicedPlan = 128;

// FP32 GEMM on the tensor cores, TF32 with a 3-term hi/lo split (tt_gemm_tc.cu).
// acc64: sum the per-K-block tensor-core partials in FP64 registers.
int gemm_tf32x3(cudaStream_t s, int M, int N, int K, double alpha, const float* A, int64_t sam,
                int64_t sak, const float* B, int64_t sbk, int64_t sbn, double beta, float* C,
                int64_t scm, int64_t scn, unsigned* status, bool acc64 = false);

// The GEMMs that form new cores in the sweeps: FP64 -> SIMT DFMA; FP32 -> the sliced
// tensor-core form when K >= 16 and its 128 x 64 tiles give every SM a CTA, else SIMT
// with compensated (Dot2) accumulation (the SIMT tiles spread small products over more
// SMs: the sliced form took the single-train QR and GEMM phases from 111 to 147 ms).  The 3xTF32
// tensor-core form is not used: it rounds every MMA result toward zero, a bias that grows
// with K and shrinks the norm of the train by about 1e-7 per sweep step, more than the
// mixed form's 1e-6 budget allows; the sliced form's tensor-core sums are exact.
template <typename T>
int gemm_core(cudaStream_t s, int M, int N, int K, double alpha, const T* A, int64_t sam, int64_t sak,
              const T* B, int64_t sbk, int64_t sbn, double beta, T* C, int64_t scm, int64_t scn,
              unsigned* status);

// The GEMM inside the Householder QR of each form: FP64 -> SIMT DFMA; FP32 -> as
// gemm_core (plain FP32 accumulation of the trailing updates took the error of 20..60-site
// trains at eps = 1e-6 from ~2e-6 to 4.6e-6: the updates need better than FP32 sums).
template <typename T>
int gemm_fast(cudaStream_t s, int M, int N, int K, double alpha, const T* A, int64_t sam, int64_t sak,
              const T* B, int64_t sbk, int64_t sbn, double beta, T* C, int64_t scm, int64_t scn,
              unsigned* status);

}  // namespace tt
