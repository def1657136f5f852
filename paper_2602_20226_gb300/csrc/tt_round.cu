// TT rounding (Section 3.2): right-to-left orthogonalisation, then the left-to-right
// sweep of truncated bond SVDs with per-bond threshold eps ||x|| / sqrt(L - 1).
//
// The output cores double as the working cores: x is copied into out (whose slots
// hold x's ranks), then every step rewrites slots in place.  Ranks never grow, so the
// slots always suffice.  All scratch is carved from the caller's workspace.
#include <chrono>
#include <type_traits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "tt_kernels.cuh"
#include "tt_qr.cuh"
#include "tt_round.cuh"
#include "tt_svd.cuh"

namespace tt {

namespace {

// Opt-in phase timer (environment variable TT_TRACE=1): synchronises the stream at
// phase boundaries and prints the wall time per phase to stderr at the end.
struct PhaseTimer {
  bool on = std::getenv("TT_TRACE") != nullptr;
  cudaStream_t s;
  std::chrono::steady_clock::time_point t0;
  double acc[8] = {0};
  const char* names[8] = {"rl_qr", "rl_formq", "rl_gemm", "lr_qr", "lr_formq", "lr_jacobi",
                          "lr_truncate", "lr_gemm"};
  explicit PhaseTimer(cudaStream_t st) : s(st) { mark(-1); }
  void mark(int phase) {
    if (!on) return;
    cudaStreamSynchronize(s);
    auto t = std::chrono::steady_clock::now();
    if (phase >= 0) acc[phase] += std::chrono::duration<double, std::milli>(t - t0).count();
    t0 = t;
  }
  ~PhaseTimer() {
    if (!on) return;
    std::fprintf(stderr, "[tt_round trace]");
    for (int i = 0; i < 8; ++i) std::fprintf(stderr, " %s=%.2fms", names[i], acc[i]);
    std::fprintf(stderr, "\n");
  }
};

// Event timing of the round's phases on the launching stream (tt_profile_enable):
// an event pair brackets every Jacobi launch, every QR (+ thin Q) and every GEMM
// group; the pairs are read back at the per-bond synchronisation that the sweep
// needs anyway, so profiling adds no extra stream synchronisation.
struct EventProfiler {
  bool on = profile_enabled();
  cudaStream_t s;
  std::vector<cudaEvent_t> ev;
  struct Rec {
    int cls;
    double nominal, executed;
  };
  std::vector<Rec> open;  // per event pair
  explicit EventProfiler(cudaStream_t st) : s(st) {}
  ~EventProfiler() {
    flush();
    for (auto e : ev) cudaEventDestroy(e);
  }
  int begin() {
    if (!on) return -1;
    const size_t i = open.size();
    while (ev.size() < 2 * (i + 1)) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      ev.push_back(e);
    }
    cudaEventRecord(ev[2 * i], s);
    open.push_back({-1, 0.0, 0.0});
    return (int)i;
  }
  // executed < 0: the executed work equals the nominal count
  void end(int i, int cls, double flops, double executed = -1.0) {
    if (!on || i < 0) return;
    cudaEventRecord(ev[2 * i + 1], s);
    open[i] = {cls, flops, executed < 0.0 ? flops : executed};
  }
  void set_executed(int i, double executed) {
    if (on && i >= 0 && i < (int)open.size()) open[i].executed = executed;
  }
  // call after the stream has been synchronised
  void flush() {
    if (!on) return;
    for (size_t i = 0; i < open.size(); ++i) {
      if (open[i].cls < 0) continue;
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]) == cudaSuccess)
        profile_add(open[i].cls, ms, open[i].nominal, open[i].executed);
    }
    open.clear();
  }
};

// FP64 bond factors of at least this rank are preconditioned by a QR of R^T before the
// Jacobi SVD (below it the extra QR costs more than the sweeps it saves)
constexpr int kPrecondMin = 48;

double qr_nominal(int m, int n) {
  const double a = std::max(m, n), b = std::min(m, n);
  return 4.0 * a * b * b - 4.0 * b * b * b / 3.0;
}

int read_back(cudaStream_t s, const void* dev, void* host, size_t bytes) {
  TT_CUDA_CHECK(cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, s));
  TT_CUDA_CHECK(cudaStreamSynchronize(s));
  return TT_OK;
}

}  // namespace

size_t round_workspace_bytes(const tt_train* x, int prec, bool batched) {
  const Dims D = dims_of(x);
  Carver c(nullptr);
  if (prec == TT_PREC_FP64) {
    Bufs<double> B;
    return carve(c, D, panel_width<double>(batched), B, batched);
  }
  Bufs<float> B;
  return carve(c, D, panel_width<float>(batched), B, batched);
}

size_t round_record_bytes(const tt_train* x) {
  const Dims D = dims_of(x);
  const size_t per = 8 * (size_t)D.S_max + 5 * (size_t)D.r_max * D.r_max + 4 * (size_t)D.r_max + 8 * 64;
  return (size_t)x->L * per * sizeof(double) + 4096;
}

template <typename T>
int round_impl(const tt_train* x, double eps, int64_t max_rank, tt_train* out, double* norm_out,
               void* ws, size_t ws_bytes, cudaStream_t s, RoundStats* stats, RoundRecord* rec) {
  const Dims D = dims_of(x);
  const int L = x->L;
  Carver c(ws);
  Bufs<T> B;
  const size_t need = carve(c, D, panel_width<T>(), B);
  if (ws_bytes < need) return fail(TT_ERR_WORKSPACE, "tt_round: workspace too small");

  std::vector<int64_t> cur(x->ranks, x->ranks + L + 1);
  std::vector<int> d(x->d, x->d + L);
  // recording for the adjoint (FP64 form only): device copies of the step's matrices
  if constexpr (!std::is_same<T, double>::value) rec = nullptr;
  auto save = [&](const void* src, size_t n) -> double* {
    double* dst = rec->take(n);
    if (dst && n) cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    return dst;
  };
  if (rec) {
    rec->rl.assign(L, RoundRecord::RL{});
    rec->lr.assign(L, RoundRecord::LR{});
  }
  T** slot = reinterpret_cast<T**>(const_cast<void**>(out->cores));
  for (int k = 0; k < L; ++k) {
    const size_t n = (size_t)cur[k] * d[k] * cur[k + 1];
    TT_CUDA_CHECK(cudaMemcpyAsync(slot[k], x->cores[k], n * sizeof(T), cudaMemcpyDeviceToDevice, s));
  }
  TT_CUDA_CHECK(cudaMemsetAsync(B.sv.status, 0, sizeof(unsigned), s));
  PhaseTimer tm(s);
  EventProfiler prof(s);

  // ---- 1. right-to-left: LQ of C_k (r_{k-1} x d r_k) as the QR of its transpose
  for (int k = L - 1; k >= 1; --k) {
    const int r0 = (int)cur[k], r1 = (int)cur[k + 1], dk = d[k];
    const int m = dk * r1, n = r0, p = std::min(m, n);
    TT_CUDA_CHECK(cudaMemcpyAsync(B.A, slot[k], (size_t)m * n * sizeof(T), cudaMemcpyDeviceToDevice, s));
    const int rows = (int)cur[k - 1] * d[k - 1];
    if (rec) {
      RoundRecord::RL& R = rec->rl[k];
      R.m = m;
      R.n = n;
      R.p = p;
      R.rows_prev = rows;
      R.dt = save(B.A, (size_t)m * n);
      R.xprev = save(slot[k - 1], (size_t)rows * n);
    }
    B.qr.ldv = m;
    int pe = prof.begin();
    TT_TRY(householder_qr<T>(s, B.A, m, n, m, B.qr));
    tm.mark(0);
    TT_TRY(form_thin_q<T>(s, B.qr, slot[k], m));  // Q^T row-major = new core [p][d][r1]
    prof.end(pe, PROF_QR, qr_nominal(m, n));
    tm.mark(1);
    TT_TRY(extract_r<T>(s, B.A, m, p, n, B.Rbuf));
    if (rec) {
      rec->rl[k].q = save(slot[k], (size_t)m * p);
      rec->rl[k].r = save(B.Rbuf, (size_t)p * n);
    }
    // C_{k-1} <- C_{k-1} R^T
    pe = prof.begin();
    TT_TRY((gemm_core<T>(s, rows, p, n, 1.0, slot[k - 1], n, 1, B.Rbuf, p, 1, 0.0, B.tmp, p, 1,
                         B.sv.status)));
    prof.end(pe, PROF_GEMM, 2.0 * rows * p * n);
    TT_CUDA_CHECK(cudaMemcpyAsync(slot[k - 1], B.tmp, (size_t)rows * p * sizeof(T),
                                  cudaMemcpyDeviceToDevice, s));
    tm.mark(2);
    cur[k] = p;
  }
  TT_TRY(frobenius_norm<T>(s, slot[0], cur[0] * d[0] * cur[1], B.sv.norm));

  // ---- 2. left-to-right truncated SVD sweep
  int total_sweeps = 0, certified_bonds = 0, refined_bonds = 0;
  if (L > 1) {
    const double delta_scale = eps / std::sqrt((double)(L - 1));
    for (int k = 0; k < L - 1; ++k) {
      const int r0 = (int)cur[k], r1 = (int)cur[k + 1];
      const int m = r0 * d[k], n = r1, p = std::min(m, n);
      const bool tall = m >= n;
      if (rec) {
        RoundRecord::LR& R = rec->lr[k];
        R.m = m;
        R.n = n;
        R.p = p;
        R.tall = tall;
        R.a = save(slot[k], (size_t)m * n);
      }
      int pe = prof.begin();
      if (tall) {
        // QR of C_k (m x n): C_k = Q R with R square (n x n); SVD of R
        TT_TRY(transpose_rm_to_cm<T>(s, slot[k], m, n, B.A));
        B.qr.ldv = m;
        TT_TRY(householder_qr<T>(s, B.A, m, n, m, B.qr));
        tm.mark(3);
        TT_TRY(form_thin_q<T>(s, B.qr, B.Q, m));
        tm.mark(4);
        // R (n x n) twice: in T for the right factor, in FP64 for the Jacobi SVD
        TT_TRY(extract_r<T>(s, B.A, m, p, n, B.Rbuf));
        if (rec) {
          rec->lr[k].q = save(B.Q, (size_t)m * p);
          rec->lr[k].r = save(B.Rbuf, (size_t)p * n);
        }
        B.sv.ldx = n;
        TT_TRY(extract_r_f64<T>(s, B.A, m, p, n, B.sv.X));
      } else {
        // wide core (m < n): LQ of C_k, i.e. the QR of C_k^T (n x m), whose column-major
        // form is C_k's own row-major memory: C_k = Rt^T Qt^T.  The left singular vectors
        // of C_k are those of the square lower-triangular Rt^T (m x m).
        TT_CUDA_CHECK(cudaMemcpyAsync(B.A, slot[k], (size_t)m * n * sizeof(T), cudaMemcpyDeviceToDevice, s));
        B.qr.ldv = n;
        TT_TRY(householder_qr<T>(s, B.A, n, m, n, B.qr));
        tm.mark(3);
        B.sv.ldx = m;
        TT_TRY(extract_rt<T>(s, B.A, n, m, m, B.sv.X));
        tm.mark(4);
      }
      prof.end(pe, PROF_QR, qr_nominal(m, n));
      pe = prof.begin();
      // No truncation is possible when sigma_min > delta: then the bond keeps its rank,
      // C_k <- Q and C_{k+1} <- R C_{k+1} represent the same tensor as the SVD factors
      // would (they differ by an orthogonal gauge), and the SVD is skipped.
      bool certified = false;
      // (the certificate subtracts p u ||R||_F with u the FP64 unit roundoff of its own
      // arithmetic, so it cannot succeed unless p u < delta / ||x||; in the mixed form it
      // certifies the stored FP32 factor, and also sigma_min > 2^-22 ||R||_F, the floor
      // below which the mixed form drops singular values)
      const double unit = 2.220446049250313e-16;
      const double cert_floor = std::is_same<T, float>::value ? kMixedSigmaFloor : 0.0;
      if (tall && (max_rank <= 0 || max_rank >= p) && 64 * (size_t)p <= 200 * 1024 && p * unit < delta_scale) {
        pe = prof.begin();
        TT_TRY(certify_full_rank(s, B.sv, B.sv.X, p, p, delta_scale, unit, cert_floor));
        prof.end(pe, PROF_CERT, (double)p * p * p / 3.0);
        int flag = 0;
        TT_TRY(read_back(s, B.sv.rank, &flag, sizeof(int)));
        prof.flush();
        certified = flag != 0;
      }
      int rn = p;
      if (certified) {
        pe = prof.begin();
        // C_k <- Q: column-major m x p is row-major p x m; transpose into row-major m x p
        TT_TRY(transpose_rm_to_cm<T>(s, B.Q, p, m, slot[k]));
        // F = R (p x n, column-major) so that C_{k+1} <- R C_{k+1} below
        TT_TRY(copy_matrix<T>(s, B.Rbuf, p, n, B.F));
        ++certified_bonds;
        if (rec) rec->lr[k].cert = true;
      } else {
        pe = prof.begin();
        int sweeps32 = 0;
        double precond_flops = 0.0;
        const bool mixed_svd = std::is_same<T, float>::value && jacobi_block_smem(p, p) <= 200 * 1024;
        if (mixed_svd) {
          // Mixed form: FP32 one-sided Jacobi (block round-robin, rotations not
          // accumulated) rotates the FP32 copy X of the factor into W = X J; sigma_j = ||W_j||
          // in FP64 and the truncation decision are FP64 (a one-sided Jacobi keeps each
          // column's rounding error relative to that column), and the kept left vectors
          // W_j / sigma_j are re-orthonormalised below.
          if (tall && p >= kPrecondMin && B.tmp64) {
            // the same preconditioning as the FP64 form, in FP64 on the FP64 copy of the
            // factor: R2^T from the QR of R^T has R's singular values and left singular
            // vectors, and the FP32 sweeps start from nearly orthogonal columns
            TT_TRY(transpose_rm_to_cm<double>(s, B.sv.X, p, p, B.tmp64));
            B.qr64.ldv = p;
            B.qr64.status = B.qr.status;
            TT_TRY(householder_qr<double>(s, B.tmp64, p, p, p, B.qr64));
            TT_TRY(extract_rt<double>(s, B.tmp64, p, p, p, B.sv.X));
            precond_flops = 4.0 * (double)p * p * p / 3.0;
          }
          TT_TRY(convert_f64_to_f32(s, B.sv.X, (int64_t)p * p, B.X32));
          TT_TRY(jacobi_block_f32(s, B.sv, B.X32, p, p, p, nullptr, p, 30));
          TT_TRY(convert_f32_to_f64(s, B.X32, (int64_t)p * p, B.sv.X));
          TT_TRY(read_back(s, B.sv.sweeps, &sweeps32, sizeof(int)));
          if (sweeps32 < 0) {
            // the FP32 sweeps did not settle: finish the (nearly diagonalised) W with FP64
            // one-sided Jacobi, which converges from there in a few sweeps
            TT_TRY(jacobi_svd(s, B.sv, p, p, jacobi_tol<double>(p), 30, delta_scale));
            ++refined_bonds;
          }
        } else {
          if (std::is_same<T, double>::value && tall && p >= kPrecondMin) {
            // preconditioning: the QR of R^T gives R = R2^T Q2^T, so R2^T has the left singular
            // vectors and the singular values of R, and one-sided Jacobi on its columns needs
            // far fewer sweeps (measured 20..36 -> 6..10 on the rank-320 bonds of the 2D
            // workload).  R^T, column-major, is R's column-major storage read row-major.
            TT_TRY(transpose_rm_to_cm<T>(s, reinterpret_cast<const T*>(B.sv.X), p, p, B.tmp));
            B.qr.ldv = p;
            TT_TRY(householder_qr<T>(s, B.tmp, p, p, p, B.qr));
            TT_TRY(extract_rt<T>(s, B.tmp, p, p, p, B.sv.X));
            precond_flops = 4.0 * (double)p * p * p / 3.0;
          } else if (tall && p >= kPrecondMin && B.tmp64) {
            // the mixed form's factors beyond the FP32 kernel's size: the same, in FP64
            TT_TRY(transpose_rm_to_cm<double>(s, B.sv.X, p, p, B.tmp64));
            B.qr64.ldv = p;
            B.qr64.status = B.qr.status;
            TT_TRY(householder_qr<double>(s, B.tmp64, p, p, p, B.qr64));
            TT_TRY(extract_rt<double>(s, B.tmp64, p, p, p, B.sv.X));
            precond_flops = 4.0 * (double)p * p * p / 3.0;
          }
          // one-sided Jacobi on the columns of the square factor X (p x p).  Pairs of columns
          // that the truncation drops in any case are left alone, except when the adjoint
          // records this run: it uses every singular pair (u_j, sigma_j) on its own, so the
          // dropped ones must be converged as well
          TT_TRY(jacobi_svd(s, B.sv, p, p, jacobi_tol<T>(p), 30, rec ? 0.0 : delta_scale));
        }
        const int pe_jacobi = pe;
        prof.end(pe, PROF_JACOBI, 12.0 * p * (double)p * p);
        tm.mark(5);
        // the FP32 Jacobi resolves singular values down to ~2^-24 sigma_1 plus the rounding
        // its rotations leave in small columns; below 2^-22 sigma_1 a column is noise
        // (nearly dependent on others), which would also defeat the Newton-Schulz step
        TT_TRY(svd_truncate(s, B.sv, p, p, delta_scale, max_rank, mixed_svd ? kMixedSigmaFloor : 0.0));
        int rk[2] = {0, 0};
        TT_TRY(read_back(s, B.sv.rank, &rk[0], 2 * sizeof(int)));  // rank, sweeps
        total_sweeps += rk[1];
        // executed work of the Jacobi: every sweep forms the three dot products of each of
        // the p (p - 1) / 2 pairs (6 p flops), and each rotation that was applied costs 6 p
        // more (the kernels count them per sweep); the mixed form's FP32 sweeps are bounded
        // by 12 p flops per pair
        if (prof.on) {
          double ex = precond_flops;
          const double pairs = 0.5 * (double)p * (p - 1);
          if (mixed_svd) {
            const int sw = sweeps32 < 0 ? 30 + std::max(rk[1], 0) : sweeps32;
            ex += 12.0 * p * pairs * std::max(sw, 0);
          } else {
            const int sw = std::max(0, std::min(rk[1], (int)SvdWork::kMaxSweeps));
            std::vector<unsigned> rots(std::max(sw, 1), 0u);
            if (sw > 0) TT_TRY(read_back(s, B.sv.rot, rots.data(), sw * sizeof(unsigned)));
            double nrot = 0.0;
            for (int q = 0; q < sw; ++q) nrot += rots[q];
            ex += 6.0 * p * (pairs * sw + nrot);
          }
          prof.set_executed(pe_jacobi, ex);
        }
        prof.flush();
        tm.mark(6);
        rn = rk[0];
        if (tm.on)
          std::fprintf(stderr, "[tt_round trace] bond %d p=%d sweeps32=%d sweeps64=%d rank=%d\n", k, p,
                       sweeps32, rk[1], rn);
        if (rn < 1 || rn > p) return fail(TT_ERR_NUMERIC, "tt_round: invalid truncation rank");
        if (rec) {
          // every left singular vector of the square factor (sorted), for the adjoint
          RoundRecord::LR& R = rec->lr[k];
          R.rn = rn;
          R.u = rec->take((size_t)p * p);
          if (R.u) TT_TRY(svd_left_vectors<double>(s, B.sv, p, p, R.u));
          R.sigma = save(B.sv.sigma, (size_t)p);
        }
        // U_r (p x r') = X[:, perm[:r']] / sigma
        pe = prof.begin();
        TT_TRY(svd_left_vectors<T>(s, B.sv, p, rn, B.vsel));
        if (mixed_svd) {
          // one Newton-Schulz step U <- U (3I - U^T U) / 2 takes the orthogonality defect
          // eta of the FP32 Jacobi's vectors to O(eta^2) (GEMMs with better-than-FP32 sums
          // keep it accurate)
          float* U = reinterpret_cast<float*>(B.vsel);
          TT_TRY((gemm_core<float>(s, rn, rn, p, 1.0, U, p, 1, U, 1, p, 0.0, B.G32, 1, rn, B.sv.status)));
          TT_TRY(newton_schulz_h(s, B.G32, rn));
          TT_TRY((gemm_core<float>(s, p, rn, rn, 1.0, U, 1, p, B.G32, 1, rn, 0.0, B.X32, 1, p, B.sv.status)));
          TT_CUDA_CHECK(cudaMemcpyAsync(U, B.X32, (size_t)p * rn * sizeof(float), cudaMemcpyDeviceToDevice, s));
        }
        if (tall) {
          // C_k <- Q U_r (m x r', row-major);  F = U_r^T R (r' x n, row-major)
          TT_TRY((gemm_core<T>(s, m, rn, p, 1.0, B.Q, 1, m, B.vsel, 1, p, 0.0, slot[k], rn, 1, B.sv.status)));
          TT_TRY((gemm_core<T>(s, rn, n, p, 1.0, B.vsel, p, 1, B.Rbuf, 1, p, 0.0, B.F, n, 1, B.sv.status)));
        } else {
          // F = U_r^T C_k (r' x n) from the original core, then C_k <- U_r (m x r', row-major)
          TT_TRY((gemm_core<T>(s, rn, n, m, 1.0, B.vsel, m, 1, slot[k], n, 1, 0.0, B.F, n, 1, B.sv.status)));
          TT_TRY(transpose_rm_to_cm<T>(s, B.vsel, rn, m, slot[k]));
        }
      }
      const int cols = d[k + 1] * (int)cur[k + 2];
      if (rec) {
        RoundRecord::LR& R = rec->lr[k];
        R.rn = rn;
        R.cols_next = cols;
        if (!certified) R.f = save(B.F, (size_t)rn * n);
        R.next = save(slot[k + 1], (size_t)n * cols);
      }
      TT_TRY((gemm_core<T>(s, rn, cols, n, 1.0, B.F, certified ? 1 : n, certified ? p : 1, slot[k + 1],
                           cols, 1, 0.0, B.tmp, cols, 1, B.sv.status)));
      TT_CUDA_CHECK(cudaMemcpyAsync(slot[k + 1], B.tmp, (size_t)rn * cols * sizeof(T),
                                    cudaMemcpyDeviceToDevice, s));
      prof.end(pe, PROF_GEMM,
               (certified ? 0.0 : (tall ? 2.0 * m * rn * p + 2.0 * rn * n * p : 2.0 * rn * n * m)) +
                   2.0 * rn * cols * n);
      tm.mark(7);
      cur[k + 1] = rn;
    }
  }
  double nrm = 0.0;
  unsigned st = 0;
  TT_TRY(read_back(s, B.sv.norm, &nrm, sizeof(double)));
  prof.flush();
  TT_TRY(read_back(s, B.sv.status, &st, sizeof(unsigned)));
  for (int k = 0; k <= L; ++k) out->ranks[k] = cur[k];
  if (norm_out) *norm_out = nrm;
  if (stats) stats->jacobi_sweeps = total_sweeps;
  if (tm.on)
    std::fprintf(stderr,
                 "[tt_round trace] jacobi sweeps total=%d, bonds certified full rank=%d, "
                 "FP32 Jacobi finished in FP64=%d\n",
                 total_sweeps, certified_bonds, refined_bonds);
  if (!std::isfinite(nrm) || (st & ST_NONFINITE)) return fail(TT_ERR_NUMERIC, "tt_round: non-finite values");
  if (st & ST_TIMEOUT) return fail(TT_ERR_TIMEOUT, "tt_round: device wait expired");
  if (st & ST_NONCONVERGED) return fail(TT_ERR_NUMERIC, "tt_round: Jacobi SVD hit its sweep cap");
  return TT_OK;
}

template int round_impl<double>(const tt_train*, double, int64_t, tt_train*, double*, void*, size_t,
                                cudaStream_t, RoundStats*, RoundRecord*);
template int round_impl<float>(const tt_train*, double, int64_t, tt_train*, double*, void*, size_t,
                               cudaStream_t, RoundStats*, RoundRecord*);

}  // namespace tt
