// GEMM entry points used inside libtt.
#pragma once

#include <algorithm>

#include "tt_common.cuh"

namespace tt {

// C = alpha * A B + beta * C with arbitrary element strides (see tt_gemm.cu).
// FP64 accumulation; beta == 0 never reads C.
template <typename TA, typename TB, typename TC>
int gemm(cudaStream_t s, int M, int N, int K, double alpha, const TA* A, int64_t sam, int64_t sak,
         const TB* B, int64_t sbk, int64_t sbn, double beta, TC* C, int64_t scm, int64_t scn);

// FP32 GEMM on the tensor cores, TF32 with a 3-term hi/lo split (tt_gemm_tc.cu).
int gemm_tf32x3(cudaStream_t s, int M, int N, int K, double alpha, const float* A, int64_t sam,
                int64_t sak, const float* B, int64_t sbk, int64_t sbn, double beta, float* C,
                int64_t scm, int64_t scn, unsigned* status);

// The GEMM of each form: FP64 -> SIMT DFMA; FP32 -> tensor cores (3xTF32).
template <typename T>
int gemm_fast(cudaStream_t s, int M, int N, int K, double alpha, const T* A, int64_t sam, int64_t sak,
              const T* B, int64_t sbk, int64_t sbn, double beta, T* C, int64_t scm, int64_t scn,
              unsigned* status);

}  // namespace tt
