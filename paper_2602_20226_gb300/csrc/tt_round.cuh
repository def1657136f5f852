// TT rounding driver.
#pragma once

#include "tt_common.cuh"

namespace tt {

struct RoundStats {
  int jacobi_sweeps = 0;
};

size_t round_workspace_bytes(const tt_train* x, int prec);

template <typename T>
int round_impl(const tt_train* x, double eps, int64_t max_rank, tt_train* out, double* norm_out,
               void* ws, size_t ws_bytes, cudaStream_t s, RoundStats* stats);

}  // namespace tt
