// Batched apply + round of many independent trains of uneven length and rank.
//
// The trains advance in lock-step: step s of the right-to-left sweep orthogonalises
// site L_i - 1 - s of every train i that still has one, step s of the left-to-right
// sweep truncates bond s of every train that has it.  Each operation of a step is ONE
// launch over all trains (one job per train, each job with its own sizes), so the
// launch count is that of a single train's sweep instead of its multiple, and the GPU
// runs hundreds of independent QR panels, bond SVDs (one CTA per train, no grid
// barriers) and GEMMs at once.  The host synchronises once per step for the data that
// sizes the next step (truncation ranks, certificate flags, FP32-sweep outcomes), read
// back for all trains with one copy each.
//
// Per train the arithmetic is that of tt_round (same QR, same truncation rule, same
// mixed-form floor), except the mixed form's bond SVD: the batched FP32 Jacobi does not
// accumulate V, and sigma and U come from its rotated columns (FP64 norms of the FP32
// columns) - a one-sided Jacobi keeps each column's rounding error relative to that
// column, which the measured errors bear out (<= 2.2e-6 at eps = 1e-6 against the
// oracle) - half the memory traffic of the V-accumulating form (8.5 s instead of 14 s of
// bond SVDs for the 512-train batch).
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <vector>

#include "tt_kernels.cuh"
#include "tt_round.cuh"

namespace tt {

namespace {

size_t align_up(size_t v) { return (v + 255) & ~size_t(255); }

// per train: the rank profile of its apply output y = W x
std::vector<int64_t> y_ranks(const tt_mpo& W, const tt_train& x) {
  std::vector<int64_t> r(x.L + 1);
  for (int k = 0; k <= x.L; ++k) r[k] = W.ranks[k] * x.ranks[k];
  return r;
}

size_t train_slice_bytes(const tt_mpo& W, const tt_train& x, int32_t prec) {
  std::vector<int64_t> r = y_ranks(W, x);
  tt_train y = x;
  y.ranks = r.data();
  return align_up(round_workspace_bytes(&y, prec, true));
}

int64_t max_y_rank(int32_t n, const tt_mpo* W, const tt_train* x) {
  int64_t m = 1;
  for (int i = 0; i < n; ++i)
    for (int k = 0; k <= x[i].L; ++k) m = std::max<int64_t>(m, W[i].ranks[k] * x[i].ranks[k]);
  return m;
}

// device region of the job arrays: enough for the update GEMMs of every panel of a QR and
// for the dozen per-step arrays, for n trains
size_t arena_bytes(int32_t n, int64_t r_max, int nb) {
  const size_t panels = (size_t)ceil_div(r_max, nb) + 1;
  // QR and thin Q: three update GEMMs per panel each
  return align_up((1u << 20) + (size_t)n * (6 * panels * sizeof(GemmJob<double, double, double>) +
                                            panels * (5 * sizeof(MapJob) + sizeof(QrJob<double>)) + 8192));
}

// results the host reads after each step, contiguous so that one copy returns them
struct Results {
  int* rank;          // [n] truncation rank / certificate flag
  int* sweeps;        // [n]
  unsigned* status;   // [n]
  double* norm;       // [n]
};

size_t results_bytes(int32_t n) { return 4 * align_up((size_t)n * 8); }

std::mutex g_pinned_mu;
char* g_pinned = nullptr;
size_t g_pinned_bytes = 0;

int pinned_staging(size_t bytes, char** out) {
  if (g_pinned_bytes < bytes) {
    if (g_pinned) TT_CUDA_CHECK(cudaFreeHost(g_pinned));
    g_pinned = nullptr;
    g_pinned_bytes = 0;
    TT_CUDA_CHECK(cudaHostAlloc(reinterpret_cast<void**>(&g_pinned), bytes, cudaHostAllocDefault));
    g_pinned_bytes = bytes;
  }
  *out = g_pinned;
  return TT_OK;
}

struct StepTimer {
  bool on = std::getenv("TT_TRACE") != nullptr;
  cudaStream_t s;
  std::chrono::steady_clock::time_point t0;
  double acc[6] = {0};
  int64_t svd_bonds = 0, sweeps32 = 0, fallbacks = 0;
  const char* names[6] = {"apply", "rl_sweep", "lr_qr", "lr_svd", "lr_gemm", "host_sync"};
  explicit StepTimer(cudaStream_t st) : s(st) { mark(-1); }
  void mark(int phase) {
    if (!on) return;
    cudaStreamSynchronize(s);
    auto t = std::chrono::steady_clock::now();
    if (phase >= 0) acc[phase] += std::chrono::duration<double, std::milli>(t - t0).count();
    t0 = t;
  }
  ~StepTimer() {
    if (!on) return;
    std::fprintf(stderr, "[tt_apply_round_batched trace]");
    for (int i = 0; i < 6; ++i) std::fprintf(stderr, " %s=%.2fms", names[i], acc[i]);
    std::fprintf(stderr, " svd_bonds=%lld fp32_sweeps=%lld fp64_finished=%lld\n", (long long)svd_bonds,
                 (long long)sweeps32, (long long)fallbacks);
  }
};

template <typename T>
struct TrainState {
  int L = 0;
  std::vector<int> d;
  std::vector<int64_t> cur;
  T** slot = nullptr;
  Bufs<T> B;
};


template <typename T>
MapJob copy_job(const T* src, T* dst, int64_t n) {
  return MapJob{src, dst, (int)n, 1, 1, 0, 1, 0, MAP_COPY};
}

// Up to four extra streams run the size classes of a step's bond SVDs side by side.
struct Lanes {
  cudaStream_t main;
  std::vector<cudaStream_t> aux;
  std::vector<cudaEvent_t> done;
  cudaEvent_t fork_ev = nullptr;
  int init(cudaStream_t s, void* const* streams, int nstreams) {
    main = s;
    for (int i = 1; i < nstreams && i <= 4; ++i) aux.push_back(as_stream(streams[i]));
    if (aux.empty()) return TT_OK;
    TT_CUDA_CHECK(cudaEventCreateWithFlags(&fork_ev, cudaEventDisableTiming));
    done.resize(aux.size(), nullptr);
    for (auto& e : done) TT_CUDA_CHECK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    return TT_OK;
  }
  ~Lanes() {
    if (fork_ev) cudaEventDestroy(fork_ev);
    for (auto e : done)
      if (e) cudaEventDestroy(e);
  }
  cudaStream_t lane(int cls) const { return aux.empty() ? main : aux[cls % aux.size()]; }
  int fork() {
    if (aux.empty()) return TT_OK;
    TT_CUDA_CHECK(cudaEventRecord(fork_ev, main));
    for (auto a : aux) TT_CUDA_CHECK(cudaStreamWaitEvent(a, fork_ev, 0));
    return TT_OK;
  }
  int join() {
    for (size_t i = 0; i < aux.size(); ++i) {
      TT_CUDA_CHECK(cudaEventRecord(done[i], aux[i]));
      TT_CUDA_CHECK(cudaStreamWaitEvent(main, done[i], 0));
    }
    return TT_OK;
  }
};

int class_of(int cs) { return cs <= 1 ? 0 : cs == 2 ? 1 : cs == 4 ? 2 : 3; }  // 8 and 16 share a lane

template <typename T>
int batched_impl(int32_t n, const tt_mpo* W, const tt_train* x, tt_train* y, double eps, int64_t max_rank,
                 tt_train* out, void* ws, size_t ws_bytes, void* const* streams, int32_t nstreams) {
  cudaStream_t s = as_stream(streams[0]);
  Lanes lanes;
  TT_TRY(lanes.init(s, streams, nstreams));
  constexpr bool kMixed = std::is_same<T, float>::value;
  const int prec = kMixed ? TT_PREC_MIXED : TT_PREC_FP64;
  const int nb = panel_width<T>(true);
  const int64_t r_max = max_y_rank(n, W, x);
  const size_t a_bytes = arena_bytes(n, r_max, nb);
  // ---- workspace: [arena | results | train slices]
  size_t need = a_bytes + results_bytes(n);
  std::vector<size_t> slice(n);
  for (int i = 0; i < n; ++i) {
    slice[i] = train_slice_bytes(W[i], x[i], prec);
    need += slice[i];
  }
  if (ws_bytes < need) return fail(TT_ERR_WORKSPACE, "tt_apply_round_batched: workspace too small");
  char* base = static_cast<char*>(ws);
  std::lock_guard<std::mutex> lock(g_pinned_mu);
  JobArena arena;
  arena.dev = base;
  arena.cap = a_bytes;
  TT_TRY(pinned_staging(a_bytes, &arena.host));
  char* rb = base + a_bytes;
  Results R;
  R.rank = reinterpret_cast<int*>(rb);
  R.sweeps = reinterpret_cast<int*>(rb + align_up((size_t)n * 8));
  R.status = reinterpret_cast<unsigned*>(rb + 2 * align_up((size_t)n * 8));
  R.norm = reinterpret_cast<double*>(rb + 3 * align_up((size_t)n * 8));
  TT_CUDA_CHECK(cudaMemsetAsync(rb, 0, results_bytes(n), s));
  StepTimer tm(s);

  std::vector<TrainState<T>> tr(n);
  char* p = rb + results_bytes(n);
  int Lmax = 0;
  for (int i = 0; i < n; ++i) {
    TrainState<T>& S = tr[i];
    S.L = x[i].L;
    Lmax = std::max(Lmax, S.L);
    S.d.assign(x[i].d, x[i].d + S.L);
    S.cur = y_ranks(W[i], x[i]);
    S.slot = reinterpret_cast<T**>(const_cast<void**>(out[i].cores));
    tt_train yi = x[i];
    yi.ranks = S.cur.data();
    Carver c(p);
    carve(c, dims_of(&yi), nb, S.B, true);
    // the host-read words of every train live in the contiguous result arrays
    S.B.sv.rank = R.rank + i;
    S.B.sv.sweeps = R.sweeps + i;
    S.B.sv.status = R.status + i;
    S.B.sv.norm = R.norm + i;
    p += slice[i];
  }
  std::vector<int> h_int(n);
  auto read_ints = [&](const int* dev) -> int {
    TT_CUDA_CHECK(cudaMemcpyAsync(h_int.data(), dev, (size_t)n * sizeof(int), cudaMemcpyDeviceToHost, s));
    TT_CUDA_CHECK(cudaStreamSynchronize(s));
    return TT_OK;
  };
  // one dense batched GEMM launch: host jobs (for the tile prefix), their device copy
  auto dense_gemm = [&](const auto& hv, const auto* dv) -> int {
    if (hv.empty()) return TT_OK;
    std::vector<int> pre(hv.size() + 1);
    const TilePlan plan = tile_prefix(hv.data(), (int)hv.size(), pre.data());
    const int* dp = arena.push(pre, s);
    if (!dp) return fail(TT_ERR_WORKSPACE, "tt_apply_round_batched: job arena full");
    return gemm_batched_dense(s, (int)hv.size(), dv, dp, plan, true, R.status);  // timeouts: train 0's word
  };
  auto step_end = [&]() -> int {
    TT_CUDA_CHECK(cudaStreamSynchronize(s));
    arena.reset();
    return TT_OK;
  };
  // ---- 1. apply, then the working copy of every core into its output slot
  for (int i = 0; i < n; ++i) TT_TRY(tt_apply_mpo(&W[i], &x[i], &y[i], s));
  {
    std::vector<MapJob> cj;
    int64_t mx = 0;
    for (int i = 0; i < n; ++i)
      for (int k = 0; k < tr[i].L; ++k) {
        const int64_t e = tr[i].cur[k] * tr[i].d[k] * tr[i].cur[k + 1];
        cj.push_back(copy_job<T>(static_cast<const T*>(y[i].cores[k]), tr[i].slot[k], e));
        mx = std::max(mx, e);
      }
    for (size_t o = 0; o < cj.size(); o += 65535) {
      std::vector<MapJob> part(cj.begin() + o, cj.begin() + std::min(cj.size(), o + 65535));
      const MapJob* dj = arena.push(part, s);
      if (!dj) return fail(TT_ERR_WORKSPACE, "tt_apply_round_batched: job arena full");
      TT_TRY((map_batched<T, T>(s, (int)part.size(), dj, mx)));
      TT_TRY(step_end());
    }
  }
  tm.mark(0);

  // ---- 2. right-to-left: LQ of C_k as the QR of its transpose, C_{k-1} <- C_{k-1} R^T
  for (int step = 0; step + 1 < Lmax; ++step) {
    std::vector<int> act;
    for (int i = 0; i < n; ++i)
      if (tr[i].L - 1 - step >= 1) act.push_back(i);
    if (act.empty()) continue;
    std::vector<MapJob> cin, rext, cout_;
    std::vector<QrJob<T>> qj;
    std::vector<GemmJob<T, T, T>> gj;
    int64_t mx_in = 0, mx_r = 0, mx_out = 0;
    for (int i : act) {
      TrainState<T>& S = tr[i];
      const int k = S.L - 1 - step;
      const int r0 = (int)S.cur[k], r1 = (int)S.cur[k + 1], dk = S.d[k];
      const int m = dk * r1, nn = r0, pp = std::min(m, nn);
      Bufs<T>& B = S.B;
      cin.push_back(copy_job<T>(S.slot[k], B.A, (int64_t)m * nn));
      mx_in = std::max<int64_t>(mx_in, (int64_t)m * nn);
      qj.push_back(QrJob<T>{B.A, m, nn, m, B.qr.tau, B.qr.tmat, B.qr.vbuf, m, B.qr.w1, B.qr.w2, S.slot[k], m,
                                  B.qr.tmat64, B.w1d, B.w2d});
      rext.push_back(MapJob{B.A, B.Rbuf, pp, nn, 1, m, 1, pp, MAP_UPPER});
      mx_r = std::max<int64_t>(mx_r, (int64_t)pp * nn);
      const int rows = (int)S.cur[k - 1] * S.d[k - 1];
      gj.push_back(GemmJob<T, T, T>{S.slot[k - 1], B.Rbuf, B.tmp, nn, 1, pp, 1, pp, 1, rows, pp, nn, 1.0, 0.0});
      cout_.push_back(copy_job<T>(B.tmp, S.slot[k - 1], (int64_t)rows * pp));
      mx_out = std::max<int64_t>(mx_out, (int64_t)rows * pp);
    }
    const int na = (int)act.size();
    const MapJob* d_cin = arena.push(cin, s);
    const QrJob<T>* d_qj = arena.push(qj, s);
    const MapJob* d_rext = arena.push(rext, s);
    const GemmJob<T, T, T>* d_gj = arena.push(gj, s);
    const MapJob* d_cout = arena.push(cout_, s);
    if (!d_cin || !d_qj || !d_rext || !d_gj || !d_cout)
      return fail(TT_ERR_WORKSPACE, "tt_apply_round_batched: job arena full");
    TT_TRY((map_batched<T, T>(s, na, d_cin, mx_in)));
    TT_TRY(householder_qr_batched<T>(s, qj, d_qj, nb, arena, R.status));
    TT_TRY(form_thin_q_batched<T>(s, qj, d_qj, nb, arena, R.status));
    TT_TRY((map_batched<T, T>(s, na, d_rext, mx_r)));
    TT_TRY(dense_gemm(gj, d_gj));
    TT_TRY((map_batched<T, T>(s, na, d_cout, mx_out)));
    for (int i : act) {
      TrainState<T>& S = tr[i];
      const int k = S.L - 1 - step;
      S.cur[k] = std::min<int64_t>(S.d[k] * S.cur[k + 1], S.cur[k]);
    }
    TT_TRY(step_end());
  }
  {
    std::vector<NormJob> nj;
    for (int i = 0; i < n; ++i)
      nj.push_back(NormJob{tr[i].slot[0], tr[i].cur[0] * tr[i].d[0] * tr[i].cur[1], R.norm + i});
    const NormJob* d_nj = arena.push(nj, s);
    if (!d_nj) return fail(TT_ERR_WORKSPACE, "tt_apply_round_batched: job arena full");
    TT_TRY(norm_batched<T>(s, n, d_nj));
    TT_TRY(step_end());
  }
  tm.mark(1);

  // ---- 3. left-to-right truncated SVD sweep
  // certificate: FP64 arithmetic in both forms (the mixed form certifies its stored FP32
  // factor, whose singular values its truncation uses, against delta and the 2^-22 floor)
  const double unit = 2.220446049250313e-16;
  for (int k = 0; k + 1 < Lmax; ++k) {
    std::vector<int> act;
    for (int i = 0; i < n; ++i)
      if (k + 1 < tr[i].L) act.push_back(i);
    if (act.empty()) continue;
    const int na = (int)act.size();
    std::vector<MapJob> cin, rext, xext;
    std::vector<QrJob<T>> qj_tall, qj_wide;
    std::vector<int> tall_idx, wide_idx;
    std::vector<int> mm(na), nn_(na), pp_(na);
    std::vector<char> tall(na);
    int64_t mx_in = 0, mx_r = 0, mx_x = 0;
    for (int a = 0; a < na; ++a) {
      TrainState<T>& S = tr[act[a]];
      Bufs<T>& B = S.B;
      const int r0 = (int)S.cur[k], r1 = (int)S.cur[k + 1];
      const int m = r0 * S.d[k], nn = r1, pp = std::min(m, nn);
      mm[a] = m;
      nn_[a] = nn;
      pp_[a] = pp;
      tall[a] = m >= nn;
      if (tall[a]) {
        cin.push_back(MapJob{S.slot[k], B.A, m, nn, nn, 1, 1, m, MAP_COPY});  // row-major -> column-major
        qj_tall.push_back(QrJob<T>{B.A, m, nn, m, B.qr.tau, B.qr.tmat, B.qr.vbuf, m, B.qr.w1, B.qr.w2, B.Q, m,
                                       B.qr.tmat64, B.w1d, B.w2d});
        tall_idx.push_back(a);
        rext.push_back(MapJob{B.A, B.Rbuf, pp, nn, 1, m, 1, pp, MAP_UPPER});
        xext.push_back(MapJob{B.A, B.sv.X, pp, nn, 1, m, 1, pp, MAP_UPPER});
      } else {
        cin.push_back(copy_job<T>(S.slot[k], B.A, (int64_t)m * nn));  // C_k^T column-major (nn x m)
        qj_wide.push_back(QrJob<T>{B.A, nn, m, nn, B.qr.tau, B.qr.tmat, B.qr.vbuf, nn, B.qr.w1, B.qr.w2, B.Q, nn,
                                       B.qr.tmat64, B.w1d, B.w2d});
        wide_idx.push_back(a);
        // X = R^T (m x m): R = upper m x m of the QR'd (nn x m) matrix
        xext.push_back(MapJob{B.A, B.sv.X, m, m, 1, nn, m, 1, MAP_UPPER});
        rext.push_back(MapJob{nullptr, nullptr, 0, 0, 0, 0, 0, 0, MAP_COPY});
      }
      B.sv.ldx = pp;
      mx_in = std::max<int64_t>(mx_in, (int64_t)m * nn);
      mx_r = std::max<int64_t>(mx_r, (int64_t)pp * nn);
      mx_x = std::max<int64_t>(mx_x, (int64_t)pp * pp);
    }
    const MapJob* d_cin = arena.push(cin, s);
    const QrJob<T>* d_qt = arena.push(qj_tall, s);
    const QrJob<T>* d_qw = arena.push(qj_wide, s);
    const MapJob* d_rext = arena.push(rext, s);
    const MapJob* d_xext = arena.push(xext, s);
    if (!d_cin || !d_qt || !d_qw || !d_rext || !d_xext)
      return fail(TT_ERR_WORKSPACE, "tt_apply_round_batched: job arena full");
    TT_TRY((map_batched<T, T>(s, na, d_cin, mx_in)));
    if (!qj_tall.empty()) {
      TT_TRY(householder_qr_batched<T>(s, qj_tall, d_qt, nb, arena, R.status));
      TT_TRY(form_thin_q_batched<T>(s, qj_tall, d_qt, nb, arena, R.status));
    }
    if (!qj_wide.empty()) TT_TRY(householder_qr_batched<T>(s, qj_wide, d_qw, nb, arena, R.status));
    TT_TRY((map_batched<T, T>(s, na, d_rext, mx_r)));
    TT_TRY((map_batched<T, double>(s, na, d_xext, mx_x)));
    tm.mark(2);

    // delta_scale = eps / sqrt(L_i - 1) differs between trains of different length: each
    // job carries its own, so one launch serves all trains of a size class
    std::vector<SvdJob> sj(na);
    for (int a = 0; a < na; ++a) {
      TrainState<T>& S = tr[act[a]];
      Bufs<T>& B = S.B;
      sj[a] = SvdJob{B.sv.X, pp_[a], pp_[a], B.X32, pp_[a], B.sv.sigma, B.sv.perm, B.sv.rank,
                     B.sv.status, B.sv.sweeps, B.sv.norm, 0, B.vsel,
                     eps / std::sqrt((double)std::max(S.L - 1, 1))};
    }
    // ---- certificate (tall bonds, max_rank not binding, when it can succeed at all:
    // it subtracts p u ||R||_F, so it needs p u < delta / ||x||)
    std::vector<char> cert(na, 0);
    {
      std::vector<SvdJob> cj;
      std::vector<int> cidx;
      for (int a = 0; a < na; ++a) {
        const double ds = eps / std::sqrt((double)std::max(tr[act[a]].L - 1, 1));
        if (tall[a] && (max_rank <= 0 || max_rank >= pp_[a]) && 64 * (size_t)pp_[a] <= 200 * 1024 &&
            pp_[a] * unit < ds) {
          cj.push_back(sj[a]);
          cidx.push_back(a);
        }
      }
      if (!cj.empty()) {
        int gmax = 0;
        for (int a : cidx) gmax = std::max(gmax, pp_[a]);
        const SvdJob* d_cj = arena.push(cj, s);
        if (!d_cj) return fail(TT_ERR_WORKSPACE, "tt_apply_round_batched: job arena full");
        TT_TRY(certify_batched(s, (int)cj.size(), d_cj, gmax, unit, kMixed ? kMixedSigmaFloor : 0.0));
        TT_TRY(read_ints(R.rank));
        for (int a : cidx) cert[a] = h_int[act[a]] != 0;
      }
    }
    // ---- bond SVDs of the others
    std::vector<int> svd_a;
    for (int a = 0; a < na; ++a)
      if (!cert[a]) svd_a.push_back(a);
    std::vector<int> rn(na);
    for (int a = 0; a < na; ++a) rn[a] = pp_[a];
    if (!svd_a.empty()) {
      std::vector<SvdJob> sv;
      int nmax = 0;
      std::vector<MapJob> conv, x32back;
      int64_t mx_pp = 0;
      for (int a : svd_a) {
        sv.push_back(sj[a]);
        nmax = std::max(nmax, pp_[a]);
        mx_pp = std::max<int64_t>(mx_pp, (int64_t)pp_[a] * pp_[a]);
        if (kMixed) {
          Bufs<T>& B = tr[act[a]].B;
          const int q = pp_[a];
          conv.push_back(MapJob{B.sv.X, B.X32, q, q, 1, q, 1, q, MAP_COPY});
          x32back.push_back(MapJob{B.X32, B.sv.X, q, q, 1, q, 1, q, MAP_COPY});
        }
      }
      const int ns = (int)sv.size();
      // jobs grouped by SVD cluster size (one stream per size class)
      auto run_grouped = [&](const std::vector<int>& qs, bool fp64_kernel, auto&& fn) -> int {
        std::vector<std::pair<int, std::vector<int>>> groups;
        for (int q : qs) {
          const int cs = svd_cluster_size(pp_[svd_a[q]], fp64_kernel);
          auto it = std::find_if(groups.begin(), groups.end(), [&](const auto& e) { return e.first == cs; });
          if (it == groups.end()) groups.push_back({cs, {q}});
          else it->second.push_back(q);
        }
        std::vector<const SvdJob*> dptr(groups.size());
        std::vector<int> gmax(groups.size(), 0);
        for (size_t g = 0; g < groups.size(); ++g) {
          std::vector<SvdJob> grp;
          for (int q : groups[g].second) {
            grp.push_back(sv[q]);
            gmax[g] = std::max(gmax[g], pp_[svd_a[q]]);
          }
          dptr[g] = arena.push(grp, s);
          if (!dptr[g]) return fail(TT_ERR_WORKSPACE, "tt_apply_round_batched: job arena full");
        }
        TT_TRY(lanes.fork());
        for (size_t g = 0; g < groups.size(); ++g) {
          const int cs = groups[g].first;
          TT_TRY(fn(lanes.lane(class_of(cs)), (int)groups[g].second.size(), dptr[g], gmax[g], cs));
        }
        return lanes.join();
      };
      std::vector<int> all_q(svd_a.size());
      for (size_t q = 0; q < svd_a.size(); ++q) all_q[q] = (int)q;
      if (kMixed) {
        const MapJob* d_conv = arena.push(conv, s);
        const MapJob* d_x32back = arena.push(x32back, s);
        if (!d_conv || !d_x32back) return fail(TT_ERR_WORKSPACE, "tt_apply_round_batched: job arena full");
        TT_TRY((map_batched<double, float>(s, ns, d_conv, mx_pp)));
        TT_TRY(run_grouped(all_q, false, [&](cudaStream_t ls, int g, const SvdJob* dg, int gm, int cs) {
          return jacobi_f32_batched(ls, g, dg, gm, 30, cs);
        }));
        TT_TRY((map_batched<float, double>(s, ns, d_x32back, mx_pp)));
        // FP32 sweeps that did not settle: finish those bonds in FP64
        TT_TRY(read_ints(R.sweeps));
        std::vector<int> fin;
        for (size_t q = 0; q < svd_a.size(); ++q) {
          const int sw = h_int[act[svd_a[q]]];
          if (sw < 0) fin.push_back((int)q);
          else tm.sweeps32 += sw;
          ++tm.svd_bonds;
        }
        tm.fallbacks += (int64_t)fin.size();
        if (!fin.empty())
          TT_TRY(run_grouped(fin, true, [&](cudaStream_t ls, int g, const SvdJob* dg, int gm, int cs) {
            return jacobi_f64_batched(ls, g, dg, gm, false, 30, cs);
          }));
      } else {
        TT_TRY(run_grouped(all_q, true, [&](cudaStream_t ls, int g, const SvdJob* dg, int gm, int cs) {
          return jacobi_f64_batched(ls, g, dg, gm, true, 30, cs);
        }));
      }
      TT_TRY(run_grouped(all_q, !kMixed, [&](cudaStream_t ls, int g, const SvdJob* dg, int gm, int) {
        return svd_truncate_batched(ls, g, dg, gm, max_rank, kMixed ? kMixedSigmaFloor : 0.0);
      }));
      TT_TRY(read_ints(R.rank));
      for (int a : svd_a) {
        rn[a] = h_int[act[a]];
        if (rn[a] < 1 || rn[a] > pp_[a]) return fail(TT_ERR_NUMERIC, "tt_apply_round_batched: invalid truncation rank");
      }
      // kept left vectors U = W[:, perm[:r]] / sigma
      std::vector<SvdJob> lv;
      int64_t mx_u = 0;
      for (int a : svd_a) {
        SvdJob J = sj[a];
        J.r = rn[a];
        lv.push_back(J);
        mx_u = std::max<int64_t>(mx_u, (int64_t)pp_[a] * rn[a]);
      }
      const SvdJob* d_lv = arena.push(lv, s);
      if (!d_lv) return fail(TT_ERR_WORKSPACE, "tt_apply_round_batched: job arena full");
      TT_TRY(svd_left_batched<T>(s, ns, d_lv, mx_u));
      if (kMixed) {
        // one Newton-Schulz step U <- U (3I - U^T U) / 2 (as in tt_round)
        std::vector<GemmJob<float, float, float>> g1, g2;
        std::vector<MapJob> h, cpy;
        int64_t mx_g = 0, mx_h = 0;
        for (int a : svd_a) {
          Bufs<T>& B = tr[act[a]].B;
          const int q = pp_[a], r = rn[a];
          float* U = reinterpret_cast<float*>(B.vsel);
          g1.push_back(GemmJob<float, float, float>{U, U, B.G32, q, 1, 1, q, 1, r, r, r, q, 1.0, 0.0});
          h.push_back(MapJob{B.G32, B.G32, r, r, 1, r, 1, r, MAP_NS});
          g2.push_back(GemmJob<float, float, float>{U, B.G32, B.X32, 1, q, 1, r, 1, q, q, r, r, 1.0, 0.0});
          cpy.push_back(copy_job<float>(B.X32, U, (int64_t)q * r));
          mx_g = std::max<int64_t>(mx_g, (int64_t)q * r);
          mx_h = std::max<int64_t>(mx_h, (int64_t)r * r);
        }
        const GemmJob<float, float, float>* d_g1 = arena.push(g1, s);
        const MapJob* d_h = arena.push(h, s);
        const GemmJob<float, float, float>* d_g2 = arena.push(g2, s);
        const MapJob* d_cpy = arena.push(cpy, s);
        if (!d_g1 || !d_h || !d_g2 || !d_cpy) return fail(TT_ERR_WORKSPACE, "tt_apply_round_batched: job arena full");
        TT_TRY(dense_gemm(g1, d_g1));
        TT_TRY((map_batched<float, float>(s, ns, d_h, mx_h)));
        TT_TRY(dense_gemm(g2, d_g2));
        TT_TRY((map_batched<float, float>(s, ns, d_cpy, mx_g)));
      }
    }
    tm.mark(3);
    // ---- new cores: C_k and the factor F that multiplies C_{k+1}
    std::vector<GemmJob<T, T, T>> ga, gb, gc;
    std::vector<MapJob> ma, mc;
    int64_t mx_a = 0, mx_c = 0;
    for (int a = 0; a < na; ++a) {
      TrainState<T>& S = tr[act[a]];
      Bufs<T>& B = S.B;
      const int m = mm[a], nn = nn_[a], q = pp_[a], r = rn[a];
      const int cols = S.d[k + 1] * (int)S.cur[k + 2];
      if (cert[a]) {
        // C_k <- Q (m x q column-major -> row-major), F = R (q x nn, column-major)
        ma.push_back(MapJob{B.Q, S.slot[k], m, q, 1, m, q, 1, MAP_COPY});
        mx_a = std::max<int64_t>(mx_a, (int64_t)m * q);
        gc.push_back(GemmJob<T, T, T>{B.Rbuf, S.slot[k + 1], B.tmp, 1, q, cols, 1, cols, 1, q, cols, nn, 1.0, 0.0});
      } else if (tall[a]) {
        // C_k <- Q U_r (m x r row-major); F = U_r^T R (r x nn row-major)
        ga.push_back(GemmJob<T, T, T>{B.Q, B.vsel, S.slot[k], 1, m, 1, q, r, 1, m, r, q, 1.0, 0.0});
        gb.push_back(GemmJob<T, T, T>{B.vsel, B.Rbuf, B.F, q, 1, 1, q, nn, 1, r, nn, q, 1.0, 0.0});
        gc.push_back(GemmJob<T, T, T>{B.F, S.slot[k + 1], B.tmp, nn, 1, cols, 1, cols, 1, r, cols, nn, 1.0, 0.0});
      } else {
        // F = U_r^T C_k (r x nn from the original core), then C_k <- U_r (row-major m x r)
        gb.push_back(GemmJob<T, T, T>{B.vsel, S.slot[k], B.F, m, 1, nn, 1, nn, 1, r, nn, m, 1.0, 0.0});
        ma.push_back(MapJob{B.vsel, S.slot[k], m, r, 1, m, r, 1, MAP_COPY});
        mx_a = std::max<int64_t>(mx_a, (int64_t)m * r);
        gc.push_back(GemmJob<T, T, T>{B.F, S.slot[k + 1], B.tmp, nn, 1, cols, 1, cols, 1, r, cols, nn, 1.0, 0.0});
      }
      mc.push_back(copy_job<T>(B.tmp, S.slot[k + 1], (int64_t)r * cols));
      mx_c = std::max<int64_t>(mx_c, (int64_t)r * cols);
    }
    // order: the F GEMMs (the wide ones read the old C_k), then the writes of the new C_k
    // (GEMM for tall bonds, copies for certified and wide ones), then C_{k+1} <- F C_{k+1}
    const GemmJob<T, T, T>* d_ga = arena.push(ga, s);
    const GemmJob<T, T, T>* d_gb = arena.push(gb, s);
    const GemmJob<T, T, T>* d_gc = arena.push(gc, s);
    const MapJob* d_ma = arena.push(ma, s);
    const MapJob* d_mc = arena.push(mc, s);
    if (!d_ga || !d_gb || !d_gc || !d_ma || !d_mc) return fail(TT_ERR_WORKSPACE, "tt_apply_round_batched: job arena full");
    TT_TRY(dense_gemm(gb, d_gb));
    TT_TRY(dense_gemm(ga, d_ga));
    if (!ma.empty()) TT_TRY((map_batched<T, T>(s, (int)ma.size(), d_ma, mx_a)));
    TT_TRY(dense_gemm(gc, d_gc));
    TT_TRY((map_batched<T, T>(s, na, d_mc, mx_c)));
    for (int a = 0; a < na; ++a) tr[act[a]].cur[k + 1] = rn[a];
    TT_TRY(step_end());
    tm.mark(4);
  }
  // ---- 4. ranks out, status words
  std::vector<unsigned> st(n);
  std::vector<double> nrm(n);
  TT_CUDA_CHECK(cudaMemcpyAsync(st.data(), R.status, (size_t)n * sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  TT_CUDA_CHECK(cudaMemcpyAsync(nrm.data(), R.norm, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, s));
  TT_CUDA_CHECK(cudaStreamSynchronize(s));
  for (int i = 0; i < n; ++i) {
    for (int k = 0; k <= tr[i].L; ++k) out[i].ranks[k] = tr[i].cur[k];
    if (!std::isfinite(nrm[i]))
      return fail(TT_ERR_NUMERIC, "tt_apply_round_batched: train " + std::to_string(i) + ": non-finite norm");
    if (st[i] & ST_NONFINITE) return fail(TT_ERR_NUMERIC, "tt_apply_round_batched: train " + std::to_string(i) + ": non-finite values");
    if (st[i] & ST_TIMEOUT) return fail(TT_ERR_TIMEOUT, "tt_apply_round_batched: device wait expired");
    if (st[i] & ST_NONCONVERGED)
      return fail(TT_ERR_NUMERIC, "tt_apply_round_batched: train " + std::to_string(i) + ": Jacobi SVD hit its sweep cap");
  }
  return TT_OK;
}

}  // namespace

size_t batched_workspace_bytes(int32_t n, const tt_mpo* W, const tt_train* x, int32_t prec) {
  const int nb = prec == TT_PREC_FP64 ? panel_width<double>(true) : panel_width<float>(true);
  size_t b = arena_bytes(n, max_y_rank(n, W, x), nb) + results_bytes(n);
  for (int i = 0; i < n; ++i) b += train_slice_bytes(W[i], x[i], prec);
  return b;
}

int apply_round_batched(int32_t n, const tt_mpo* W, const tt_train* x, tt_train* y, double eps,
                        int64_t max_rank, int32_t prec, tt_train* out, void* ws, size_t ws_bytes,
                        void* const* streams, int32_t nstreams) {
  if (prec == TT_PREC_FP64) return batched_impl<double>(n, W, x, y, eps, max_rank, out, ws, ws_bytes, streams, nstreams);
  return batched_impl<float>(n, W, x, y, eps, max_rank, out, ws, ws_bytes, streams, nstreams);
}

}  // namespace tt
