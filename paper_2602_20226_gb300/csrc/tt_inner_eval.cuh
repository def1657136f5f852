// Inner product, evaluation and their adjoints.
#pragma once

#include "tt_common.cuh"

namespace tt {

template <typename T>
struct EvalParams {
  int L;
  int rmax;
  const T* g[TT_MAX_SITES];
  int d[TT_MAX_SITES];
  int r[TT_MAX_SITES + 1];
};

size_t inner_workspace_bytes(const tt_train* x, const tt_train* y);
template <typename TX, typename TY>
int inner_impl(const tt_train* x, const tt_train* y, double* out, void* ws, size_t ws_bytes,
               cudaStream_t s);
template <typename TX, typename TY>
int inner_backward_impl(const tt_train* x, const tt_train* y, double dout, tt_train* dx,
                        tt_train* dy, void* ws, size_t ws_bytes, cudaStream_t s);

// tt_inner with its scratch in a fixed device array (tt_noalloc.cu)
int inner_noalloc(const tt_train* x, const tt_train* y, double* out, cudaStream_t s);

template <typename T>
int eval_impl(const tt_train* x, const uint8_t* digits, int64_t n, void* values, cudaStream_t s,
              unsigned* status_dev);
size_t eval_backward_workspace_bytes(const tt_train* x, int64_t n);
template <typename T>
int eval_backward_impl(const tt_train* x, const uint8_t* digits, int64_t n, const void* dvalues,
                       tt_train* dx, void* ws, size_t ws_bytes, cudaStream_t s);

}  // namespace tt
