// Batched apply + round over many independent trains of uneven length and rank.
//
// A host-side scheduler: `nstreams` worker threads, each bound to one caller stream
// and one slice of the caller's workspace, pull trains from a shared queue ordered by
// nominal work (largest first, the longest-processing-time rule) and run tt_apply_mpo
// then tt_round on their stream.  One train's sweep is a sequential chain of small,
// latency-bound launches; running many chains at once fills the GPU.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <numeric>
#include <thread>
#include <vector>

#include "tt_round.cuh"

namespace tt {

namespace {

double nominal_work(const tt_mpo& W, const tt_train& x) {
  // pre-round bond ranks a_k r_k; rounding costs ~ sum_k n_k^3
  double w = 0.0;
  for (int k = 0; k < x.L; ++k) {
    const double n = (double)W.ranks[k + 1] * (double)x.ranks[k + 1];
    w += n * n * n + 1.0;
  }
  return w;
}

size_t align_up(size_t v) { return (v + 255) & ~size_t(255); }

}  // namespace

size_t batched_slice_bytes(int32_t n, const tt_mpo* W, const tt_train* x, int32_t prec) {
  size_t m = 0;
  for (int i = 0; i < n; ++i) {
    std::vector<int64_t> r(x[i].L + 1);
    for (int k = 0; k <= x[i].L; ++k) r[k] = W[i].ranks[k] * x[i].ranks[k];
    tt_train y = x[i];
    y.ranks = r.data();
    m = std::max(m, round_workspace_bytes(&y, prec));
  }
  return align_up(m);
}

int apply_round_batched(int32_t n, const tt_mpo* W, const tt_train* x, tt_train* y, double eps,
                        int64_t max_rank, int32_t prec, tt_train* out, void* ws, size_t ws_bytes,
                        void* const* streams, int32_t nstreams) {
  const size_t slice = batched_slice_bytes(n, W, x, prec);
  if (ws_bytes < slice * (size_t)nstreams)
    return fail(TT_ERR_WORKSPACE, "tt_apply_round_batched: workspace too small");
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::vector<double> work(n);
  for (int i = 0; i < n; ++i) work[i] = nominal_work(W[i], x[i]);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work[a] > work[b]; });

  std::atomic<int> next{0};
  std::atomic<int> first_error{TT_OK};
  std::vector<std::string> errors(nstreams);
  int dev = 0;
  TT_CUDA_CHECK(cudaGetDevice(&dev));
  auto worker = [&](int t) {
    cudaSetDevice(dev);
    cudaStream_t s = as_stream(streams[t]);
    char* base = static_cast<char*>(ws) + slice * (size_t)t;
    for (;;) {
      if (first_error.load() != TT_OK) return;
      const int q = next.fetch_add(1);
      if (q >= n) return;
      const int i = order[q];
      int code = tt_apply_mpo(&W[i], &x[i], &y[i], s);
      if (code == TT_OK)
        code = tt_round(&y[i], eps, max_rank, prec, &out[i], nullptr, base, slice, s);
      if (code != TT_OK) {
        int expected = TT_OK;
        if (first_error.compare_exchange_strong(expected, code))
          errors[t] = "train " + std::to_string(i) + ": " + tt_last_error();
        return;
      }
    }
  };
  std::vector<std::thread> pool;
  for (int t = 0; t < nstreams; ++t) pool.emplace_back(worker, t);
  for (auto& th : pool) th.join();
  const int code = first_error.load();
  if (code != TT_OK) {
    for (auto& e : errors)
      if (!e.empty()) return fail(code, "tt_apply_round_batched: " + e);
    return fail(code, "tt_apply_round_batched failed");
  }
  for (int t = 0; t < nstreams; ++t) TT_CUDA_CHECK(cudaStreamSynchronize(as_stream(streams[t])));
  return TT_OK;
}

}  // namespace tt
