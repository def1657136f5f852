// C ABI of libtt: host-side validation, dispatch by dtype, error plumbing.
// Nothing is enqueued before all arguments have been checked.  No exception leaves
// an entry point.
#include <atomic>
#include <mutex>
#include <cmath>
#include <cstdio>
#include <exception>
#include <string>
#include <vector>

#include "tt_gemm.cuh"
#include "tt_inner_eval.cuh"
#include "tt_kernels.cuh"
#include "tt_round.cuh"

namespace tt {

namespace {
thread_local std::string g_last_error;
std::atomic<unsigned long long> g_launches{0};
}  // namespace

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

namespace {
std::atomic<bool> g_prof_on{false};
std::mutex g_prof_mu;
double g_prof_ms[PROF_CLASSES] = {0}, g_prof_flops[PROF_CLASSES] = {0}, g_prof_exec[PROF_CLASSES] = {0};
uint64_t g_prof_n[PROF_CLASSES] = {0};
}  // namespace

bool profile_enabled() { return g_prof_on.load(std::memory_order_relaxed); }

void profile_add(int cls, double ms, double flops, double executed) {
  if (cls < 0 || cls >= PROF_CLASSES) return;
  std::lock_guard<std::mutex> g(g_prof_mu);
  g_prof_ms[cls] += ms;
  g_prof_flops[cls] += flops;
  g_prof_exec[cls] += executed;
  g_prof_n[cls] += 1;
}

void set_error(const std::string& msg) { g_last_error = msg; }

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int num_sms() {
  // cached for the last device asked about; the count is stored before the device tag, so a
  // thread that sees the tag sees its count
  static std::atomic<int> dev_cached{-1}, sms{0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (dev != dev_cached.load()) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) v = 1;
    sms.store(v);
    dev_cached.store(dev);
    return v;
  }
  return sms.load();
}

namespace {

constexpr int64_t kMaxCoreElems = (int64_t)1 << 31;

int check_dims(int L, const int32_t* d, const char* what) {
  if (L < 1 || L > TT_MAX_SITES)
    return fail(TT_ERR_UNSUPPORTED, std::string(what) + ": L must be in [1, TT_MAX_SITES]");
  if (!d) return fail(TT_ERR_ARG, std::string(what) + ": d is NULL");
  for (int k = 0; k < L; ++k)
    if (d[k] < 1 || d[k] > TT_MAX_MODE)
      return fail(TT_ERR_UNSUPPORTED, std::string(what) + ": mode size out of [1, TT_MAX_MODE]");
  return TT_OK;
}

int check_ranks(int L, const int64_t* r, const int32_t* d, int mode_mult, const char* what) {
  if (!r) return fail(TT_ERR_ARG, std::string(what) + ": ranks is NULL");
  if (r[0] != 1 || r[L] != 1) return fail(TT_ERR_SHAPE, std::string(what) + ": boundary ranks must be 1");
  for (int k = 0; k <= L; ++k)
    if (r[k] < 1 || r[k] > (1 << 24)) return fail(TT_ERR_SHAPE, std::string(what) + ": rank out of range");
  for (int k = 0; k < L; ++k) {
    int64_t e = r[k] * (int64_t)d[k] * r[k + 1];
    for (int u = 1; u < mode_mult; ++u) e *= d[k];
    if (e >= kMaxCoreElems) return fail(TT_ERR_UNSUPPORTED, std::string(what) + ": core has >= 2^31 elements");
  }
  return TT_OK;
}

int check_cores(int L, void* const* cores, const char* what, bool allow_null_entries = false) {
  if (!cores) return fail(TT_ERR_ARG, std::string(what) + ": cores is NULL");
  if (!allow_null_entries)
    for (int k = 0; k < L; ++k)
      if (!cores[k]) return fail(TT_ERR_ARG, std::string(what) + ": a core pointer is NULL");
  return TT_OK;
}

int check_train(const tt_train* x, const char* what, bool ranks_valid = true) {
  if (!x) return fail(TT_ERR_ARG, std::string(what) + " is NULL");
  TT_TRY(check_dims(x->L, x->d, what));
  if (x->dtype != TT_F64 && x->dtype != TT_F32) return fail(TT_ERR_DTYPE, std::string(what) + ": bad dtype");
  if (ranks_valid) TT_TRY(check_ranks(x->L, x->ranks, x->d, 1, what));
  else if (!x->ranks) return fail(TT_ERR_ARG, std::string(what) + ": ranks is NULL");
  return check_cores(x->L, x->cores, what);
}

int check_same_modes(const tt_train* a, const int32_t* d, int L, const char* what) {
  if (a->L != L) return fail(TT_ERR_SHAPE, std::string(what) + ": length mismatch");
  for (int k = 0; k < L; ++k)
    if (a->d[k] != d[k]) return fail(TT_ERR_SHAPE, std::string(what) + ": mode mismatch");
  return TT_OK;
}

template <typename F>
int guarded(F&& f) {
  try {
    return f();
  } catch (const std::exception& e) {
    return fail(TT_ERR_ARG, std::string("internal error: ") + e.what());
  } catch (...) {
    return fail(TT_ERR_ARG, "internal error");
  }
}

template <typename T>
int apply_typed(const tt_mpo* W, const tt_train* x, tt_train* y, cudaStream_t s) {
  ApplyParams<T> P;
  P.L = x->L;
  P.row_start[0] = 0;
  for (int k = 0; k < x->L; ++k) {
    ApplySite<T>& S = P.site[k];
    S.w = static_cast<const T*>(W->cores[k]);
    S.g = static_cast<const T*>(x->cores[k]);
    S.y = static_cast<T*>(y->cores[k]);
    S.d = x->d[k];
    S.a0 = (int)W->ranks[k];
    S.a1 = (int)W->ranks[k + 1];
    S.r0 = (int)x->ranks[k];
    S.r1 = (int)x->ranks[k + 1];
    P.row_start[k + 1] = P.row_start[k] + (long long)S.a0 * S.r0 * S.d;
  }
  return launch_apply<T>(s, P);
}

template <typename T>
int hadamard_typed(const tt_train* x, const tt_train* y, tt_train* z, cudaStream_t s) {
  HadamardParams<T> P;
  P.L = x->L;
  P.row_start[0] = 0;
  for (int k = 0; k < x->L; ++k) {
    HadamardSite<T>& S = P.site[k];
    S.x = static_cast<const T*>(x->cores[k]);
    S.y = static_cast<const T*>(y->cores[k]);
    S.z = static_cast<T*>(z->cores[k]);
    S.d = x->d[k];
    S.r0 = (int)x->ranks[k];
    S.r1 = (int)x->ranks[k + 1];
    S.s0 = (int)y->ranks[k];
    S.s1 = (int)y->ranks[k + 1];
    P.row_start[k + 1] = P.row_start[k] + (long long)S.r0 * S.s0 * S.d;
  }
  return launch_hadamard<T>(s, P);
}

template <typename T>
int apply_bwd_typed(const tt_mpo* W, const tt_train* x, const tt_train* dy, tt_mpo* dW,
                    tt_train* dx, cudaStream_t s) {
  ApplyBwdParams<T> P;
  P.L = x->L;
  P.row_start[0] = 0;
  P.wblk_start[0] = 0;
  for (int k = 0; k < x->L; ++k) {
    ApplyBwdSite<T>& S = P.site[k];
    S.w = static_cast<const T*>(W->cores[k]);
    S.g = static_cast<const T*>(x->cores[k]);
    S.dy = static_cast<const T*>(dy->cores[k]);
    S.dg = dx ? static_cast<T*>(dx->cores[k]) : nullptr;
    S.dw = dW ? static_cast<T*>(dW->cores[k]) : nullptr;
    S.d = x->d[k];
    S.a0 = (int)W->ranks[k];
    S.a1 = (int)W->ranks[k + 1];
    S.r0 = (int)x->ranks[k];
    S.r1 = (int)x->ranks[k + 1];
    P.row_start[k + 1] = P.row_start[k] + (long long)S.r0 * S.d;
    P.wblk_start[k + 1] = P.wblk_start[k] + (long long)S.a0 * S.d * S.a1;
  }
  return launch_apply_bwd<T>(s, P, dx != nullptr, dW != nullptr);
}

template <typename T>
int hadamard_bwd_typed(const tt_train* x, const tt_train* y, const tt_train* dz, tt_train* dx,
                       tt_train* dy, cudaStream_t s) {
  HadamardBwdParams<T> P;
  P.L = x->L;
  P.xrow_start[0] = 0;
  P.yrow_start[0] = 0;
  for (int k = 0; k < x->L; ++k) {
    HadamardBwdSite<T>& S = P.site[k];
    S.x = static_cast<const T*>(x->cores[k]);
    S.y = static_cast<const T*>(y->cores[k]);
    S.dz = static_cast<const T*>(dz->cores[k]);
    S.dx = dx ? static_cast<T*>(dx->cores[k]) : nullptr;
    S.dy = dy ? static_cast<T*>(dy->cores[k]) : nullptr;
    S.d = x->d[k];
    S.r0 = (int)x->ranks[k];
    S.r1 = (int)x->ranks[k + 1];
    S.s0 = (int)y->ranks[k];
    S.s1 = (int)y->ranks[k + 1];
    P.xrow_start[k + 1] = P.xrow_start[k] + (long long)S.r0 * S.d * S.r1;
    P.yrow_start[k + 1] = P.yrow_start[k] + (long long)S.s0 * S.d;
  }
  return launch_hadamard_bwd<T>(s, P, dx != nullptr, dy != nullptr);
}

int validate_mpo(const tt_mpo* W, const tt_train* x) {
  if (!W) return fail(TT_ERR_ARG, "W is NULL");
  TT_TRY(check_dims(W->L, W->d, "W"));
  if (W->L != x->L) return fail(TT_ERR_SHAPE, "W: length mismatch");
  for (int k = 0; k < x->L; ++k)
    if (W->d[k] != x->d[k]) return fail(TT_ERR_SHAPE, "W: mode mismatch");
  if (W->dtype != x->dtype) return fail(TT_ERR_DTYPE, "W: dtype differs from x");
  TT_TRY(check_ranks(W->L, W->ranks, W->d, 2, "W"));
  return check_cores(W->L, W->cores, "W");
}

int validate_out(const tt_train* y, const tt_train* x, const char* what) {
  if (!y) return fail(TT_ERR_ARG, std::string(what) + " is NULL");
  if (!y->d || !y->ranks) return fail(TT_ERR_ARG, std::string(what) + ": d or ranks is NULL");
  TT_TRY(check_same_modes(y, x->d, x->L, what));
  if (y->dtype != x->dtype) return fail(TT_ERR_DTYPE, std::string(what) + ": dtype differs");
  return check_cores(y->L, y->cores, what);
}

}  // namespace
}  // namespace tt

using namespace tt;

extern "C" {

const char* tt_last_error(void) { return g_last_error.c_str(); }

const char* tt_version(void) { return "libtt 0.1 (sm_103a)"; }

uint64_t tt_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

void tt_profile_enable(int32_t on) {
  std::lock_guard<std::mutex> g(g_prof_mu);
  for (int c = 0; c < PROF_CLASSES; ++c) g_prof_ms[c] = g_prof_flops[c] = g_prof_exec[c] = 0.0, g_prof_n[c] = 0;
  g_prof_on.store(on != 0);
}

int tt_profile_read(int32_t cls, double* ms, double* nominal_flops, uint64_t* count) {
  if (cls < 0 || cls >= PROF_CLASSES) return fail(TT_ERR_ARG, "tt_profile_read: bad class");
  std::lock_guard<std::mutex> g(g_prof_mu);
  if (ms) *ms = g_prof_ms[cls];
  if (nominal_flops) *nominal_flops = g_prof_flops[cls];
  if (count) *count = g_prof_n[cls];
  return TT_OK;
}

int tt_profile_read_executed(int32_t cls, double* executed_flops) {
  if (cls < 0 || cls >= PROF_CLASSES) return fail(TT_ERR_ARG, "tt_profile_read_executed: bad class");
  std::lock_guard<std::mutex> g(g_prof_mu);
  if (executed_flops) *executed_flops = g_prof_exec[cls];
  return TT_OK;
}

int tt_apply_mpo(const tt_mpo* W, const tt_train* x, tt_train* y, void* stream) {
  return guarded([&]() -> int {
    TT_TRY(check_train(x, "x"));
    TT_TRY(validate_mpo(W, x));
    TT_TRY(validate_out(y, x, "y"));
    std::vector<int64_t> r(x->L + 1);
    for (int k = 0; k <= x->L; ++k) r[k] = W->ranks[k] * x->ranks[k];
    for (int k = 0; k < x->L; ++k)
      if (r[k] * x->d[k] * r[k + 1] >= kMaxCoreElems)
        return fail(TT_ERR_UNSUPPORTED, "tt_apply_mpo: output core has >= 2^31 elements");
    for (int k = 0; k <= x->L; ++k) y->ranks[k] = r[k];
    g_last_error.clear();
    return x->dtype == TT_F64 ? apply_typed<double>(W, x, y, as_stream(stream))
                              : apply_typed<float>(W, x, y, as_stream(stream));
  });
}

int tt_hadamard(const tt_train* x, const tt_train* y, tt_train* z, void* stream) {
  return guarded([&]() -> int {
    TT_TRY(check_train(x, "x"));
    TT_TRY(check_train(y, "y"));
    TT_TRY(check_same_modes(y, x->d, x->L, "y"));
    if (y->dtype != x->dtype) return fail(TT_ERR_DTYPE, "y: dtype differs from x");
    TT_TRY(validate_out(z, x, "z"));
    std::vector<int64_t> r(x->L + 1);
    for (int k = 0; k <= x->L; ++k) r[k] = x->ranks[k] * y->ranks[k];
    for (int k = 0; k < x->L; ++k)
      if (r[k] * x->d[k] * r[k + 1] >= kMaxCoreElems)
        return fail(TT_ERR_UNSUPPORTED, "tt_hadamard: output core has >= 2^31 elements");
    for (int k = 0; k <= x->L; ++k) z->ranks[k] = r[k];
    g_last_error.clear();
    return x->dtype == TT_F64 ? hadamard_typed<double>(x, y, z, as_stream(stream))
                              : hadamard_typed<float>(x, y, z, as_stream(stream));
  });
}

size_t tt_round_workspace_size(const tt_train* x, int32_t prec) {
  if (check_train(x, "x") != TT_OK) return 0;
  return round_workspace_bytes(x, prec);
}

int tt_round(const tt_train* x, double eps, int64_t max_rank, int32_t prec, tt_train* out,
             double* norm_out, void* workspace, size_t ws_bytes, void* stream) {
  return guarded([&]() -> int {
    TT_TRY(check_train(x, "x"));
    TT_TRY(validate_out(out, x, "out"));
    if (!(eps >= 0.0) || !std::isfinite(eps)) return fail(TT_ERR_ARG, "tt_round: eps must be finite and >= 0");
    if (prec == TT_PREC_FP64 && x->dtype != TT_F64)
      return fail(TT_ERR_DTYPE, "tt_round: TT_PREC_FP64 needs TT_F64 cores");
    if (prec == TT_PREC_MIXED && x->dtype != TT_F32)
      return fail(TT_ERR_DTYPE, "tt_round: TT_PREC_MIXED needs TT_F32 cores");
    if (prec != TT_PREC_FP64 && prec != TT_PREC_MIXED) return fail(TT_ERR_ARG, "tt_round: bad prec");
    if (!workspace) return fail(TT_ERR_WORKSPACE, "tt_round: workspace is NULL");
    g_last_error.clear();
    if (prec == TT_PREC_FP64)
      return round_impl<double>(x, eps, max_rank, out, norm_out, workspace, ws_bytes, as_stream(stream), nullptr);
    return round_impl<float>(x, eps, max_rank, out, norm_out, workspace, ws_bytes, as_stream(stream), nullptr);
  });
}

size_t tt_round_backward_workspace_size(const tt_train* x) {
  if (check_train(x, "x") != TT_OK) return 0;
  return round_backward_workspace_bytes(x);
}

int tt_round_backward(const tt_train* x, double eps, int64_t max_rank, const tt_train* dout, tt_train* dx,
                      void* workspace, size_t ws_bytes, void* stream) {
  return guarded([&]() -> int {
    TT_TRY(check_train(x, "x"));
    TT_TRY(check_train(dout, "dout"));
    TT_TRY(check_train(dx, "dx"));
    if (x->dtype != TT_F64 || dout->dtype != TT_F64 || dx->dtype != TT_F64)
      return fail(TT_ERR_DTYPE, "tt_round_backward: x, dout and dx must be TT_F64 (the FP64 form)");
    TT_TRY(check_same_modes(dout, x->d, x->L, "dout"));
    TT_TRY(check_same_modes(dx, x->d, x->L, "dx"));
    for (int k = 0; k <= x->L; ++k)
      if (dx->ranks[k] != x->ranks[k]) return fail(TT_ERR_SHAPE, "tt_round_backward: dx must have x's ranks");
    if (!(eps >= 0.0) || !std::isfinite(eps)) return fail(TT_ERR_ARG, "tt_round_backward: eps must be finite and >= 0");
    if (!workspace) return fail(TT_ERR_WORKSPACE, "tt_round_backward: workspace is NULL");
    g_last_error.clear();
    return round_backward_impl(x, eps, max_rank, dout, dx, workspace, ws_bytes, as_stream(stream));
  });
}

size_t tt_inner_workspace_size(const tt_train* x, const tt_train* y) {
  if (check_train(x, "x") != TT_OK || check_train(y, "y") != TT_OK) return 0;
  return inner_workspace_bytes(x, y);
}

int tt_inner(const tt_train* x, const tt_train* y, double* out, void* workspace, size_t ws_bytes,
             void* stream) {
  return guarded([&]() -> int {
    TT_TRY(check_train(x, "x"));
    TT_TRY(check_train(y, "y"));
    TT_TRY(check_same_modes(y, x->d, x->L, "y"));
    if (y->dtype != x->dtype) return fail(TT_ERR_DTYPE, "y: dtype differs from x");
    if (!out) return fail(TT_ERR_ARG, "tt_inner: out is NULL");
    if (!workspace) return fail(TT_ERR_WORKSPACE, "tt_inner: workspace is NULL");
    g_last_error.clear();
    return x->dtype == TT_F64
               ? inner_impl<double, double>(x, y, out, workspace, ws_bytes, as_stream(stream))
               : inner_impl<float, float>(x, y, out, workspace, ws_bytes, as_stream(stream));
  });
}

int tt_inner_noalloc(const tt_train* x, const tt_train* y, double* out, void* stream) {
  return guarded([&]() -> int {
    TT_TRY(check_train(x, "x"));
    TT_TRY(check_train(y, "y"));
    TT_TRY(check_same_modes(y, x->d, x->L, "y"));
    if (y->dtype != x->dtype) return fail(TT_ERR_DTYPE, "y: dtype differs from x");
    if (!out) return fail(TT_ERR_ARG, "tt_inner_noalloc: out is NULL");
    g_last_error.clear();
    return inner_noalloc(x, y, out, as_stream(stream));
  });
}

int tt_eval(const tt_train* x, const uint8_t* digits, int64_t n, void* values, void* stream) {
  return guarded([&]() -> int {
    TT_TRY(check_train(x, "x"));
    if (n < 0) return fail(TT_ERR_ARG, "tt_eval: n < 0");
    if (n > 0 && (!digits || !values)) return fail(TT_ERR_ARG, "tt_eval: digits or values is NULL");
    g_last_error.clear();
    return x->dtype == TT_F64 ? eval_impl<double>(x, digits, n, values, as_stream(stream), nullptr)
                              : eval_impl<float>(x, digits, n, values, as_stream(stream), nullptr);
  });
}

int tt_apply_mpo_backward(const tt_mpo* W, const tt_train* x, const tt_train* dy, tt_mpo* dW,
                          tt_train* dx, void* stream) {
  return guarded([&]() -> int {
    TT_TRY(check_train(x, "x"));
    TT_TRY(validate_mpo(W, x));
    TT_TRY(check_train(dy, "dy"));
    for (int k = 0; k <= x->L; ++k)
      if (dy->ranks[k] != W->ranks[k] * x->ranks[k]) return fail(TT_ERR_SHAPE, "dy: ranks must be a_k r_k");
    if (dy->dtype != x->dtype) return fail(TT_ERR_DTYPE, "dy: dtype differs from x");
    if (dx) {
      TT_TRY(validate_out(dx, x, "dx"));
      for (int k = 0; k <= x->L; ++k)
        if (dx->ranks[k] != x->ranks[k]) return fail(TT_ERR_SHAPE, "dx: ranks differ from x");
    }
    if (dW) {
      if (dW->L != x->L || dW->dtype != x->dtype) return fail(TT_ERR_SHAPE, "dW: shape or dtype differs from W");
      TT_TRY(check_cores(dW->L, dW->cores, "dW"));
    }
    g_last_error.clear();
    return x->dtype == TT_F64 ? apply_bwd_typed<double>(W, x, dy, dW, dx, as_stream(stream))
                              : apply_bwd_typed<float>(W, x, dy, dW, dx, as_stream(stream));
  });
}

int tt_hadamard_backward(const tt_train* x, const tt_train* y, const tt_train* dz, tt_train* dx,
                         tt_train* dy, void* stream) {
  return guarded([&]() -> int {
    TT_TRY(check_train(x, "x"));
    TT_TRY(check_train(y, "y"));
    TT_TRY(check_same_modes(y, x->d, x->L, "y"));
    TT_TRY(check_train(dz, "dz"));
    for (int k = 0; k <= x->L; ++k)
      if (dz->ranks[k] != x->ranks[k] * y->ranks[k]) return fail(TT_ERR_SHAPE, "dz: ranks must be r_k s_k");
    if (y->dtype != x->dtype || dz->dtype != x->dtype) return fail(TT_ERR_DTYPE, "dtype mismatch");
    if (dx) TT_TRY(validate_out(dx, x, "dx"));
    if (dy) TT_TRY(validate_out(dy, y, "dy"));
    g_last_error.clear();
    return x->dtype == TT_F64 ? hadamard_bwd_typed<double>(x, y, dz, dx, dy, as_stream(stream))
                              : hadamard_bwd_typed<float>(x, y, dz, dx, dy, as_stream(stream));
  });
}

int tt_inner_backward(const tt_train* x, const tt_train* y, double dout, tt_train* dx,
                      tt_train* dy, void* workspace, size_t ws_bytes, void* stream) {
  return guarded([&]() -> int {
    TT_TRY(check_train(x, "x"));
    TT_TRY(check_train(y, "y"));
    TT_TRY(check_same_modes(y, x->d, x->L, "y"));
    if (y->dtype != x->dtype) return fail(TT_ERR_DTYPE, "y: dtype differs from x");
    if (dx) TT_TRY(validate_out(dx, x, "dx"));
    if (dy) TT_TRY(validate_out(dy, y, "dy"));
    if (!workspace) return fail(TT_ERR_WORKSPACE, "tt_inner_backward: workspace is NULL");
    g_last_error.clear();
    return x->dtype == TT_F64
               ? inner_backward_impl<double, double>(x, y, dout, dx, dy, workspace, ws_bytes, as_stream(stream))
               : inner_backward_impl<float, float>(x, y, dout, dx, dy, workspace, ws_bytes, as_stream(stream));
  });
}

size_t tt_eval_backward_workspace_size(const tt_train* x, int64_t n) {
  if (check_train(x, "x") != TT_OK || n < 0) return 0;
  return eval_backward_workspace_bytes(x, n);
}

int tt_eval_backward(const tt_train* x, const uint8_t* digits, int64_t n, const void* dvalues,
                     tt_train* dx, void* workspace, size_t ws_bytes, void* stream) {
  return guarded([&]() -> int {
    TT_TRY(check_train(x, "x"));
    TT_TRY(validate_out(dx, x, "dx"));
    if (n < 0) return fail(TT_ERR_ARG, "tt_eval_backward: n < 0");
    if (n > 0 && (!digits || !dvalues)) return fail(TT_ERR_ARG, "tt_eval_backward: digits or dvalues is NULL");
    if (n > 0 && !workspace) return fail(TT_ERR_WORKSPACE, "tt_eval_backward: workspace is NULL");
    g_last_error.clear();
    return x->dtype == TT_F64
               ? eval_backward_impl<double>(x, digits, n, dvalues, dx, workspace, ws_bytes, as_stream(stream))
               : eval_backward_impl<float>(x, digits, n, dvalues, dx, workspace, ws_bytes, as_stream(stream));
  });
}

size_t tt_apply_round_batched_workspace_size(int32_t n, const tt_mpo* W, const tt_train* x,
                                             int32_t prec, int32_t nstreams) {
  if (n <= 0 || !W || !x || nstreams < 1) return 0;
  for (int i = 0; i < n; ++i)
    if (check_train(&x[i], "x") != TT_OK || validate_mpo(&W[i], &x[i]) != TT_OK) return 0;
  if (prec != TT_PREC_FP64 && prec != TT_PREC_MIXED) return 0;
  return batched_workspace_bytes(n, W, x, prec);
}

int tt_apply_round_batched(int32_t n, const tt_mpo* W, const tt_train* x, tt_train* y, double eps,
                           int64_t max_rank, int32_t prec, tt_train* out, void* workspace,
                           size_t ws_bytes, void* const* streams, int32_t nstreams) {
  return guarded([&]() -> int {
    if (n < 0) return fail(TT_ERR_ARG, "tt_apply_round_batched: n < 0");
    if (n == 0) return TT_OK;
    if (!W || !x || !y || !out) return fail(TT_ERR_ARG, "tt_apply_round_batched: NULL descriptor array");
    if (nstreams < 1 || !streams) return fail(TT_ERR_ARG, "tt_apply_round_batched: no streams");
    if (!workspace) return fail(TT_ERR_WORKSPACE, "tt_apply_round_batched: workspace is NULL");
    if (!(eps >= 0.0) || !std::isfinite(eps)) return fail(TT_ERR_ARG, "tt_apply_round_batched: eps must be finite and >= 0");
    if (prec != TT_PREC_FP64 && prec != TT_PREC_MIXED) return fail(TT_ERR_ARG, "tt_apply_round_batched: bad prec");
    for (int i = 0; i < n; ++i) {
      if (prec == TT_PREC_FP64 && x[i].dtype != TT_F64)
        return fail(TT_ERR_DTYPE, "tt_apply_round_batched: TT_PREC_FP64 needs TT_F64 cores");
      if (prec == TT_PREC_MIXED && x[i].dtype != TT_F32)
        return fail(TT_ERR_DTYPE, "tt_apply_round_batched: TT_PREC_MIXED needs TT_F32 cores");
    }
    for (int i = 0; i < n; ++i) {
      TT_TRY(check_train(&x[i], "x"));
      TT_TRY(validate_mpo(&W[i], &x[i]));
      TT_TRY(validate_out(&y[i], &x[i], "y"));
      TT_TRY(validate_out(&out[i], &x[i], "out"));
    }
    g_last_error.clear();
    return apply_round_batched(n, W, x, y, eps, max_rank, prec, out, workspace, ws_bytes, streams, nstreams);
  });
}

int tt_gemm_f32(int32_t M, int32_t N, int32_t K, double alpha, const float* A, int64_t sam,
                int64_t sak, const float* B, int64_t sbk, int64_t sbn, double beta, float* C,
                int64_t scm, int64_t scn, void* stream) {
  return guarded([&]() -> int {
    if (M < 0 || N < 0 || K < 0) return fail(TT_ERR_ARG, "tt_gemm_f32: negative size");
    if ((M > 0 && N > 0) && (!C || (K > 0 && (!A || !B)))) return fail(TT_ERR_ARG, "tt_gemm_f32: NULL operand");
    g_last_error.clear();
    return gemm_tf32x3(as_stream(stream), M, N, K, alpha, A, sam, sak, B, sbk, sbn, beta, C, scm, scn,
                       nullptr);
  });
}

int tt_gemm_f32_sliced(int32_t M, int32_t N, int32_t K, double alpha, const float* A, int64_t sam,
                       int64_t sak, const float* B, int64_t sbk, int64_t sbn, double beta, float* C,
                       int64_t scm, int64_t scn, void* stream) {
  return guarded([&]() -> int {
    if (M < 0 || N < 0 || K < 0) return fail(TT_ERR_ARG, "tt_gemm_f32_sliced: negative size");
    if ((M > 0 && N > 0) && (!C || (K > 0 && (!A || !B))))
      return fail(TT_ERR_ARG, "tt_gemm_f32_sliced: NULL operand");
    g_last_error.clear();
    return gemm_sliced(as_stream(stream), M, N, K, alpha, A, sam, sak, B, sbk, sbn, beta, C, scm, scn, nullptr);
  });
}

}  // extern "C"
