// TT rounding (Section 3.2): right-to-left orthogonalisation, then the left-to-right
// sweep of truncated bond SVDs with per-bond threshold eps ||x|| / sqrt(L - 1).
//
// The output cores double as the working cores: x is copied into out (whose slots
// hold x's ranks), then every step rewrites slots in place.  Ranks never grow, so the
// slots always suffice.  All scratch is carved from the caller's workspace.
#include <cmath>
#include <vector>

#include "tt_kernels.cuh"
#include "tt_qr.cuh"
#include "tt_round.cuh"
#include "tt_svd.cuh"

namespace tt {

namespace {

struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* b) : base(static_cast<char*>(b)) {}
  template <typename U>
  U* take(size_t n) {
    off = (off + 255) & ~size_t(255);
    U* p = base ? reinterpret_cast<U*>(base + off) : nullptr;
    off += n * sizeof(U);
    return p;
  }
};

struct Dims {
  int L = 0;
  int64_t S_max = 1;  // largest core (elements)
  int64_t r_max = 1;  // largest rank
};

Dims dims_of(const tt_train* x) {
  Dims D;
  D.L = x->L;
  for (int k = 0; k < x->L; ++k) {
    D.S_max = std::max<int64_t>(D.S_max, x->ranks[k] * (int64_t)x->d[k] * x->ranks[k + 1]);
    D.r_max = std::max<int64_t>(D.r_max, std::max(x->ranks[k], x->ranks[k + 1]));
  }
  return D;
}

template <typename T>
struct Bufs {
  T *A = nullptr, *Q = nullptr, *tmp = nullptr, *Rbuf = nullptr, *vsel = nullptr, *F = nullptr;
  QrWork<T> qr;
  SvdWork sv;
};

template <typename T>
size_t carve(Carver& c, const Dims& D, int nb, Bufs<T>& B) {
  B.A = c.take<T>(D.S_max);
  B.Q = c.take<T>(D.S_max);
  B.tmp = c.take<T>(D.S_max);
  B.qr.nb = nb;
  B.qr.vbuf = c.take<T>(D.S_max);
  B.qr.tau = c.take<T>(D.r_max + 32);
  B.qr.tmat = c.take<T>((size_t)nb * nb * (ceil_div(D.r_max, nb) + 1));
  B.qr.w1 = c.take<T>((size_t)nb * D.r_max);
  B.qr.w2 = c.take<T>((size_t)nb * D.r_max);
  B.Rbuf = c.take<T>((size_t)D.r_max * D.r_max);
  B.vsel = c.take<T>((size_t)D.r_max * D.r_max);
  B.F = c.take<T>((size_t)D.r_max * D.r_max);
  B.sv.X = c.take<double>((size_t)D.r_max * D.r_max);
  B.sv.V = c.take<double>((size_t)D.r_max * D.r_max);
  B.sv.sigma = c.take<double>(D.r_max);
  B.sv.perm = c.take<int>(D.r_max);
  B.sv.rank = c.take<int>(1);
  B.sv.bar = c.take<unsigned>(2);
  B.sv.rot = c.take<unsigned>(SvdWork::kMaxSweeps);
  B.sv.status = c.take<unsigned>(1);
  B.sv.sweeps = c.take<int>(1);
  B.sv.norm = c.take<double>(1);
  return c.off + 256;
}

template <typename T>
int panel_width() {
  return sizeof(T) == 8 ? 16 : 32;
}

template <typename T>
double jacobi_tol(int nrow) {
  // columns are treated as orthogonal once |x_a . x_b| <= tol ||x_a|| ||x_b||
  return std::sqrt((double)std::max(nrow, 1)) * 2.220446049250313e-16;
}

int read_back(cudaStream_t s, const void* dev, void* host, size_t bytes) {
  TT_CUDA_CHECK(cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, s));
  TT_CUDA_CHECK(cudaStreamSynchronize(s));
  return TT_OK;
}

}  // namespace

size_t round_workspace_bytes(const tt_train* x, int prec) {
  const Dims D = dims_of(x);
  Carver c(nullptr);
  if (prec == TT_PREC_FP64) {
    Bufs<double> B;
    return carve(c, D, panel_width<double>(), B);
  }
  Bufs<float> B;
  return carve(c, D, panel_width<float>(), B);
}

template <typename T>
int round_impl(const tt_train* x, double eps, int64_t max_rank, tt_train* out, double* norm_out,
               void* ws, size_t ws_bytes, cudaStream_t s, RoundStats* stats) {
  const Dims D = dims_of(x);
  const int L = x->L;
  Carver c(ws);
  Bufs<T> B;
  const size_t need = carve(c, D, panel_width<T>(), B);
  if (ws_bytes < need) return fail(TT_ERR_WORKSPACE, "tt_round: workspace too small");

  std::vector<int64_t> cur(x->ranks, x->ranks + L + 1);
  std::vector<int> d(x->d, x->d + L);
  T** slot = reinterpret_cast<T**>(const_cast<void**>(out->cores));
  for (int k = 0; k < L; ++k) {
    const size_t n = (size_t)cur[k] * d[k] * cur[k + 1];
    TT_CUDA_CHECK(cudaMemcpyAsync(slot[k], x->cores[k], n * sizeof(T), cudaMemcpyDeviceToDevice, s));
  }
  TT_CUDA_CHECK(cudaMemsetAsync(B.sv.status, 0, sizeof(unsigned), s));

  // ---- 1. right-to-left: LQ of C_k (r_{k-1} x d r_k) as the QR of its transpose
  for (int k = L - 1; k >= 1; --k) {
    const int r0 = (int)cur[k], r1 = (int)cur[k + 1], dk = d[k];
    const int m = dk * r1, n = r0, p = std::min(m, n);
    TT_CUDA_CHECK(cudaMemcpyAsync(B.A, slot[k], (size_t)m * n * sizeof(T), cudaMemcpyDeviceToDevice, s));
    B.qr.ldv = m;
    TT_TRY(householder_qr<T>(s, B.A, m, n, m, B.qr));
    TT_TRY(form_thin_q<T>(s, B.qr, slot[k], m));  // Q^T row-major = new core [p][d][r1]
    TT_TRY(extract_r<T>(s, B.A, m, p, n, B.Rbuf));
    const int rows = (int)cur[k - 1] * d[k - 1];
    // C_{k-1} <- C_{k-1} R^T
    TT_TRY((gemm<T, T, T>(s, rows, p, n, 1.0, slot[k - 1], n, 1, B.Rbuf, p, 1, 0.0, B.tmp, p, 1)));
    TT_CUDA_CHECK(cudaMemcpyAsync(slot[k - 1], B.tmp, (size_t)rows * p * sizeof(T),
                                  cudaMemcpyDeviceToDevice, s));
    cur[k] = p;
  }
  TT_TRY(frobenius_norm<T>(s, slot[0], cur[0] * d[0] * cur[1], B.sv.norm));

  // ---- 2. left-to-right truncated SVD sweep
  int total_sweeps = 0;
  if (L > 1) {
    const double delta_scale = eps / std::sqrt((double)(L - 1));
    for (int k = 0; k < L - 1; ++k) {
      const int r0 = (int)cur[k], r1 = (int)cur[k + 1];
      const int m = r0 * d[k], n = r1, p = std::min(m, n);
      TT_TRY(transpose_rm_to_cm<T>(s, slot[k], m, n, B.A));
      B.qr.ldv = m;
      TT_TRY(householder_qr<T>(s, B.A, m, n, m, B.qr));
      TT_TRY(form_thin_q<T>(s, B.qr, B.Q, m));
      B.sv.ldx = n;
      B.sv.ldv = p;
      TT_TRY(extract_rt<T>(s, B.A, m, p, n, B.sv.X));
      TT_TRY(jacobi_svd(s, B.sv, n, p, jacobi_tol<T>(n), 30));
      TT_TRY(svd_truncate(s, B.sv, n, p, delta_scale, max_rank));
      int rk[2] = {0, 0};
      TT_TRY(read_back(s, B.sv.rank, &rk[0], sizeof(int)));
      TT_TRY(read_back(s, B.sv.sweeps, &rk[1], sizeof(int)));
      total_sweeps += rk[1];
      const int rn = rk[0];
      if (rn < 1 || rn > p) return fail(TT_ERR_NUMERIC, "tt_round: invalid truncation rank");
      TT_TRY(svd_gather<T>(s, B.sv, n, p, rn, B.vsel, B.F));
      // C_k <- Q V[:, perm[:r']]   (m x r', row-major)
      TT_TRY((gemm<T, T, T>(s, m, rn, p, 1.0, B.Q, 1, m, B.vsel, 1, p, 0.0, slot[k], rn, 1)));
      // C_{k+1} <- W[:, perm[:r']]^T C_{k+1}
      const int cols = d[k + 1] * (int)cur[k + 2];
      TT_TRY((gemm<T, T, T>(s, rn, cols, n, 1.0, B.F, n, 1, slot[k + 1], cols, 1, 0.0, B.tmp, cols, 1)));
      TT_CUDA_CHECK(cudaMemcpyAsync(slot[k + 1], B.tmp, (size_t)rn * cols * sizeof(T),
                                    cudaMemcpyDeviceToDevice, s));
      cur[k + 1] = rn;
    }
  }
  double nrm = 0.0;
  unsigned st = 0;
  TT_TRY(read_back(s, B.sv.norm, &nrm, sizeof(double)));
  TT_TRY(read_back(s, B.sv.status, &st, sizeof(unsigned)));
  for (int k = 0; k <= L; ++k) out->ranks[k] = cur[k];
  if (norm_out) *norm_out = nrm;
  if (stats) stats->jacobi_sweeps = total_sweeps;
  if (!std::isfinite(nrm) || (st & ST_NONFINITE)) return fail(TT_ERR_NUMERIC, "tt_round: non-finite values");
  if (st & ST_TIMEOUT) return fail(TT_ERR_TIMEOUT, "tt_round: device wait expired");
  if (st & ST_NONCONVERGED) return fail(TT_ERR_NUMERIC, "tt_round: Jacobi SVD hit its sweep cap");
  return TT_OK;
}

template int round_impl<double>(const tt_train*, double, int64_t, tt_train*, double*, void*, size_t,
                                cudaStream_t, RoundStats*);
template int round_impl<float>(const tt_train*, double, int64_t, tt_train*, double*, void*, size_t,
                               cudaStream_t, RoundStats*);

}  // namespace tt
