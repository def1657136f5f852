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

}  // namespace tt
