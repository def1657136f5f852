// Diagnostics of the device-side failure handling (no counterpart in the paper).
//
// tt_debug_wait_expiry runs the library's bounded wait (bounded_wait_ge, the wait of the
// dataflow Jacobi SVDs) on a flag that nothing ever sets: the wait gives up after the
// given number of polls, raises ST_TIMEOUT in the status word and the kernel returns, so
// the host sees TT_ERR_TIMEOUT with the context intact.  No trap, no fault, no endless loop.
#include "tt_common.cuh"

namespace tt {
namespace {

__global__ void wait_expiry_kernel(const unsigned* flag, unsigned* status, long long limit, unsigned* done) {
  if (threadIdx.x == 0) {
    const bool ok = bounded_wait_ge(flag, 1u, status, limit);
    *done = ok ? 1u : 2u;
  }
}

}  // namespace
}  // namespace tt

using namespace tt;

extern "C" int tt_debug_wait_expiry(int64_t poll_limit, void* scratch, void* stream) {
  if (!scratch) return fail(TT_ERR_ARG, "tt_debug_wait_expiry: scratch is NULL");
  if (poll_limit < 1 || poll_limit > (int64_t)kWaitPolls)
    return fail(TT_ERR_ARG, "tt_debug_wait_expiry: poll_limit must be in [1, 2^24]");
  cudaStream_t s = as_stream(stream);
  unsigned* w = static_cast<unsigned*>(scratch);  // [0] flag, [1] status, [2] outcome
  TT_CUDA_CHECK(cudaMemsetAsync(w, 0, 3 * sizeof(unsigned), s));
  wait_expiry_kernel<<<1, 32, 0, s>>>(w, w + 1, (long long)poll_limit, w + 2);
  TT_LAUNCH_CHECK();
  unsigned h[3] = {0, 0, 0};
  TT_CUDA_CHECK(cudaMemcpyAsync(h, w, sizeof(h), cudaMemcpyDeviceToHost, s));
  TT_CUDA_CHECK(cudaStreamSynchronize(s));
  if (h[1] & ST_TIMEOUT) return fail(TT_ERR_TIMEOUT, "tt_debug_wait_expiry: the bounded wait expired");
  return TT_OK;
}
