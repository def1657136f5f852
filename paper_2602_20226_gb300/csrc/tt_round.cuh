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

size_t batched_slice_bytes(int32_t n, const tt_mpo* W, const tt_train* x, int32_t prec);
int apply_round_batched(int32_t n, const tt_mpo* W, const tt_train* x, tt_train* y, double eps,
                        int64_t max_rank, int32_t prec, tt_train* out, void* ws, size_t ws_bytes,
                        void* const* streams, int32_t nstreams);

}  // namespace tt
