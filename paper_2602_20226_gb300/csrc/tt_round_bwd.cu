// Adjoint of TT rounding in FP64 (tt_round_backward).
//
// The forward sweeps are run again exactly as tt_round runs them (round_impl, recording the
// factors of every step), so the output cores - and the gauge that the caller's cotangent
// refers to - are the ones tt_round returned.  Then the two sweeps are reversed:
//
//  * left-to-right bonds, last to first.  A bond maps the current core A (m x n) to the
//    output core B and the factor F that multiplies the next core, C_{k+1} <- F C_{k+1}.
//    Certified bonds are a thin QR, B = Q, F = R: the QR adjoint
//        M = R dR^T - dQ^T Q,  dA = (dQ + Q copyltu(M)) R^{-T}.
//    SVD bonds take the leading r' left singular vectors, B = U_r, F = B^T A: with u all left
//    singular vectors of A (u = Q U_R from the square factor's SVD), dU = [dB, 0],
//    P = u^T dB, M = [P 0] - [P 0]^T, G_ij = M_ij / (s_j^2 - s_i^2) (0 for near-degenerate
//    pairs and for zero singular values j),
//        dA = u G u^T A + (dB - u P) S_r^{-2} (u^T A)[:r'] + B dF,
//    the singular-vector perturbation formula with S V^T written as u^T A, so no right
//    singular vectors are needed.
//  * right-to-left steps, first to last: D_{k-1} = x_{k-1} R_k^T gives dx_{k-1} and dR_k,
//    and the QR adjoint of D_k^T = Q_k R_k (tall, or wide: a = Q [R1 R2]) gives dD_k.
//
// All arithmetic is FP64 on the library's strided GEMM and three small kernels (the
// antisymmetric / copyltu combinations and a triangular solve).
#include <cmath>
#include <vector>

#include "tt_gemm.cuh"
#include "tt_kernels.cuh"
#include "tt_round.cuh"

namespace tt {

namespace {

// C (n x n, cm) = tril(M) + tril(M, -1)^T
__global__ void copyltu_kernel(const double* M, int n, double* C) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  const int i = (int)(e % n), j = (int)(e / n);
  C[e] = i >= j ? M[i + (int64_t)j * n] : M[j + (int64_t)i * n];
}

// G (k x k, cm) from P (k x rn, cm): M_ij = P_ij [j < rn] - P_ji [i < rn];
// G_ij = M_ij / (s_j^2 - s_i^2), 0 on the diagonal, for |s_j^2 - s_i^2| <= tiny and for s_j = 0.
__global__ void svd_adj_g_kernel(const double* P, int k, int rn, const double* s, double tiny, double* G) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)k * k) return;
  const int i = (int)(e % k), j = (int)(e / k);
  double m = 0.0;
  if (j < rn) m += P[i + (int64_t)j * k];
  if (i < rn) m -= P[j + (int64_t)i * k];
  const double si = s[i], sj = s[j];
  const double diff = sj * sj - si * si;
  G[e] = (i == j || sj == 0.0 || fabs(diff) <= tiny) ? 0.0 : m / diff;
}

// X (rows x n, element (i, j) at X[i*sxr + j*sxc]) <- X R^{-T} for the upper-triangular
// R (n x n, cm, ld ldr): each row x solves R x^T = x_old^T by back substitution.  One warp
// per row; the solved entries stay in shared memory.
constexpr int kTrsmWarps = 4;
__global__ void __launch_bounds__(32 * kTrsmWarps) trsm_rt_kernel(double* X, int rows, int n, int64_t sxr, int64_t sxc,
                                                                  const double* R, int ldr) {
  extern __shared__ double zs[];  // [kTrsmWarps][n]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int row = blockIdx.x * kTrsmWarps + w;
  if (row >= rows) return;  // whole warps leave; no block barrier below
  double* z = zs + (int64_t)w * n;
  double* xr = X + (int64_t)row * sxr;
  for (int j = lane; j < n; j += 32) z[j] = xr[(int64_t)j * sxc];
  __syncwarp();
  for (int i = n - 1; i >= 0; --i) {
    double part = 0.0;
    for (int j = i + 1 + lane; j < n; j += 32) part = fma(R[i + (int64_t)j * ldr], z[j], part);
    part = warp_sum(part);
    if (lane == 0) z[i] = (z[i] - part) / R[i + (int64_t)i * ldr];
    __syncwarp();
  }
  for (int j = lane; j < n; j += 32) xr[(int64_t)j * sxc] = z[j];
}

// A factor is treated as singular (no derivative: the bond rank of x exceeds the rank of its
// unfolding) when its smallest diagonal entry is below 1e-13 of its largest.
__global__ void diag_check_kernel(const double* R, int n, int ldr, unsigned* status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double lo = INFINITY, hi = 0.0;
  for (int i = 0; i < n; ++i) {
    const double v = fabs(R[i + (int64_t)i * ldr]);
    lo = fmin(lo, v);
    hi = fmax(hi, v);
  }
  if (!(lo > 1e-13 * hi)) atomicOr(status, (unsigned)ST_NONFINITE);
}

// X (rows x cols, cm) *= d_j per column (d from s: 1 / s_j^2 for s_j > 0, else 0)
__global__ void scale_cols_inv2_kernel(double* X, int rows, int cols, const double* s) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)rows * cols) return;
  const int j = (int)(e / rows);
  const double sj = s[j];
  X[e] = sj > 0.0 ? X[e] / (sj * sj) : 0.0;
}

__global__ void finite_kernel(const double* X, int64_t n, unsigned* status) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(X[e])) {
      atomicOr(status, (unsigned)ST_NONFINITE);
      return;
    }
}

unsigned blocks_for(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), 1 << 20)); }

inline int gemm64(cudaStream_t s, int M, int N, int K, double alpha, const double* A, int64_t sam, int64_t sak,
                  const double* B, int64_t sbk, int64_t sbn, double beta, double* C, int64_t scm, int64_t scn) {
  return gemm<double, double, double>(s, M, N, K, alpha, A, sam, sak, B, sbk, sbn, beta, C, scm, scn);
}

struct Scratch {
  char* base;
  size_t cap, off = 0;
  double* take(size_t n) {
    off = (off + 255) & ~size_t(255);
    if (off + n * sizeof(double) > cap) return nullptr;
    double* p = reinterpret_cast<double*>(base + off);
    off += n * sizeof(double);
    return p;
  }
};

__global__ void add_strided_kernel(double* Y, int rows, int cols, int64_t syr, int64_t syc, const double* X, int64_t sxr,
                                   int64_t sxc, double alpha) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)rows * cols) return;
  const int i = (int)(e % rows), j = (int)(e / rows);
  Y[i * syr + j * syc] += alpha * X[i * sxr + j * sxc];
}

int add_strided(cudaStream_t s, double* Y, int rows, int cols, int64_t syr, int64_t syc, const double* X, int64_t sxr,
                int64_t sxc, double alpha = 1.0) {
  if ((int64_t)rows * cols <= 0) return TT_OK;
  add_strided_kernel<<<blocks_for((int64_t)rows * cols), 256, 0, s>>>(Y, rows, cols, syr, syc, X, sxr, sxc, alpha);
  TT_LAUNCH_CHECK();
  return TT_OK;
}

int trsm_rt(cudaStream_t s, double* X, int rows, int n, int64_t sxr, int64_t sxc, const double* R, int ldr,
            unsigned* status) {
  if (rows <= 0 || n <= 0) return TT_OK;
  diag_check_kernel<<<1, 32, 0, s>>>(R, n, ldr, status);
  TT_LAUNCH_CHECK();
  const size_t smem = (size_t)kTrsmWarps * n * sizeof(double);
  if (smem > 200 * 1024) return fail(TT_ERR_UNSUPPORTED, "tt_round_backward: factor too large for the solve");
  static std::atomic<int> configured{-1};
  int dev = 0;
  TT_CUDA_CHECK(cudaGetDevice(&dev));
  if (configured != dev) {
    TT_CUDA_CHECK(cudaFuncSetAttribute(trsm_rt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    configured = dev;
  }
  trsm_rt_kernel<<<(unsigned)ceil_div(rows, kTrsmWarps), 32 * kTrsmWarps, smem, s>>>(X, rows, n, sxr, sxc, R, ldr);
  TT_LAUNCH_CHECK();
  return TT_OK;
}

// Thin-QR adjoint, tall or wide.  a = q r with a m x n (cm), q m x p cm, r p x n cm (p = min).
// dq: m x p (element (i, j) at dq[i*sqr + j*sqc]); dr: p x n cm.  dA written m x n cm.
int qr_adjoint(cudaStream_t s, int m, int n, const double* a, const double* q, const double* r, const double* dq,
               int64_t sqr, int64_t sqc, double* dr, double* dA, Scratch& sc, unsigned* status) {
  const int p = std::min(m, n);
  const size_t mark = sc.off;
  double* dqc = sc.take((size_t)m * p);  // dq, column-major (plus the wide correction)
  double* M = sc.take((size_t)p * p);
  double* C = sc.take((size_t)p * p);
  if (!dqc || !M || !C) return fail(TT_ERR_WORKSPACE, "tt_round_backward: workspace too small");
  TT_CUDA_CHECK(cudaMemsetAsync(dqc, 0, (size_t)m * p * sizeof(double), s));
  TT_TRY(add_strided(s, dqc, m, p, 1, m, dq, sqr, sqc));
  if (m < n) {
    // wide: a = [x y], r = [r1 r2]; dy = q dr2, and x = q r1 with dq + y dr2^T
    const int n2 = n - m;
    TT_TRY(gemm64(s, m, n2, m, 1.0, q, 1, m, dr + (int64_t)m * p, 1, p, 0.0, dA + (int64_t)m * m, 1, m));
    TT_TRY(gemm64(s, m, m, n2, 1.0, a + (int64_t)m * m, 1, m, dr + (int64_t)m * p, p, 1, 1.0, dqc, 1, m));
  }
  // square / tall part on the first p columns: M = r1 dr1^T - dq^T q
  TT_TRY(gemm64(s, p, p, p, 1.0, r, 1, p, dr, p, 1, 0.0, M, 1, p));
  TT_TRY(gemm64(s, p, p, m, -1.0, dqc, m, 1, q, 1, m, 1.0, M, 1, p));
  copyltu_kernel<<<blocks_for((int64_t)p * p), 256, 0, s>>>(M, p, C);
  TT_LAUNCH_CHECK();
  // dA[:, :p] = (dq + q C) r1^{-T}
  TT_CUDA_CHECK(cudaMemcpyAsync(dA, dqc, (size_t)m * p * sizeof(double), cudaMemcpyDeviceToDevice, s));
  TT_TRY(gemm64(s, m, p, p, 1.0, q, 1, m, C, 1, p, 1.0, dA, 1, m));
  TT_TRY(trsm_rt(s, dA, m, p, 1, m, r, p, status));
  sc.off = mark;
  return TT_OK;
}

}  // namespace

namespace {
size_t core_bytes(const tt_train* x, int k) {
  return ((size_t)x->ranks[k] * x->d[k] * x->ranks[k + 1] * sizeof(double) + 255) & ~size_t(255);
}
size_t scratch_doubles(const Dims& D) { return 8 * (size_t)D.S_max + 10 * (size_t)D.r_max * D.r_max + 256; }
}  // namespace

size_t round_backward_workspace_bytes(const tt_train* x) {
  const Dims D = dims_of(x);
  Carver c(nullptr);
  Bufs<double> B;
  const size_t fwd = carve(c, D, panel_width<double>(), B);
  // forward workspace + output slots of the recomputed rounding + the record + the
  // cotangents of the right-to-left output cores + scratch
  size_t slots = 0;
  for (int k = 0; k < x->L; ++k) slots += core_bytes(x, k);
  return fwd + 2 * slots + round_record_bytes(x) + scratch_doubles(D) * sizeof(double) + 8192;
}

int round_backward_impl(const tt_train* x, double eps, int64_t max_rank, const tt_train* dout, tt_train* dx,
                        void* ws, size_t ws_bytes, cudaStream_t s) {
  if (ws_bytes < round_backward_workspace_bytes(x)) return fail(TT_ERR_WORKSPACE, "tt_round_backward: workspace too small");
  const int L = x->L;
  const Dims D = dims_of(x);
  char* base = static_cast<char*>(ws);
  size_t off = 0;
  auto carve_bytes = [&](size_t b) {
    off = (off + 255) & ~size_t(255);
    char* p = base + off;
    off += b;
    return p;
  };
  // ---- 1. the forward rounding again, recording every step
  Carver c0(nullptr);
  Bufs<double> B0;
  const size_t fwd = carve(c0, D, panel_width<double>(), B0);
  void* fws = carve_bytes(fwd);
  std::vector<void*> oslot(L);
  for (int k = 0; k < L; ++k) oslot[k] = carve_bytes((size_t)x->ranks[k] * x->d[k] * x->ranks[k + 1] * sizeof(double));
  std::vector<int64_t> oranks(L + 1);
  tt_train out = *x;
  out.ranks = oranks.data();
  out.cores = oslot.data();
  RoundRecord rec;
  rec.cap = round_record_bytes(x);
  rec.base = carve_bytes(rec.cap);
  std::vector<double*> dcrl(L, nullptr);  // cotangents of the right-to-left output cores
  for (int k = 0; k < L; ++k) dcrl[k] = reinterpret_cast<double*>(carve_bytes(core_bytes(x, k)));
  Scratch sc{carve_bytes(scratch_doubles(D) * sizeof(double)), scratch_doubles(D) * sizeof(double)};
  if (off > ws_bytes) return fail(TT_ERR_WORKSPACE, "tt_round_backward: workspace too small");
  double nrm = 0.0;
  TT_TRY(round_impl<double>(x, eps, max_rank, &out, &nrm, fws, fwd, s, nullptr, &rec));
  if (rec.overflow) return fail(TT_ERR_WORKSPACE, "tt_round_backward: record arena too small");
  for (int k = 0; k <= L; ++k)
    if (dout->ranks[k] != oranks[k])
      return fail(TT_ERR_SHAPE, "tt_round_backward: dout's ranks differ from those of round(x)");
  unsigned* status = reinterpret_cast<unsigned*>(sc.take(1));
  if (!status) return fail(TT_ERR_WORKSPACE, "tt_round_backward: workspace too small");
  TT_CUDA_CHECK(cudaMemsetAsync(status, 0, sizeof(double), s));
  const double guard = 1e-13;

  // ---- 2. reverse of the left-to-right sweep: g = cotangent of the current core k + 1
  const size_t dmax = (size_t)D.S_max;
  double* g = sc.take(dmax);
  double* g2 = sc.take(dmax);
  if (!g || !g2) return fail(TT_ERR_WORKSPACE, "tt_round_backward: workspace too small");
  {
    const size_t n_last = (size_t)oranks[L - 1] * x->d[L - 1] * oranks[L];
    TT_CUDA_CHECK(cudaMemcpyAsync(g, dout->cores[L - 1], n_last * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  for (int k = L - 2; k >= 0; --k) {
    const RoundRecord::LR& R = rec.lr[k];
    const int m = R.m, n = R.n, p = R.p, rn = R.rn, cols = R.cols_next;
    const size_t mark = sc.off;
    double* dF = sc.take((size_t)std::max(rn, p) * n);  // rn x n row-major (cert: p x n cm)
    double* dA = g2;                                     // m x n row-major
    if (!dF) return fail(TT_ERR_WORKSPACE, "tt_round_backward: workspace too small");
    const double* dOutk = static_cast<const double*>(dout->cores[k]);  // m x rn row-major
    if (R.cert) {
      // B = Q (m x p cm = the output core, row-major m x p), F = R (p x n cm)
      // dF (p x n cm) = g (p x cols rm) next^T (cols x n): element (i, j) at i + j p
      TT_TRY(gemm64(s, p, n, cols, 1.0, g, cols, 1, R.next, 1, cols, 0.0, dF, 1, p));
      // dC_rl[k+1] (n x cols rm) = F^T g = R^T (n x p) g (p x cols)
      TT_TRY(gemm64(s, n, cols, p, 1.0, R.r, p, 1, g, cols, 1, 0.0, dcrl[k + 1], cols, 1));
      // QR adjoint of A (m x n row-major = cm n x m transposed; the QR was of A as m x n):
      // dq = dout_k (m x p row-major: element (i, j) at i * p + j), dr = dF
      double* dAc = sc.take((size_t)m * n);
      double* acm = sc.take((size_t)m * n);
      if (!dAc || !acm) return fail(TT_ERR_WORKSPACE, "tt_round_backward: workspace too small");
      // a as column-major (the QR factorised it so): a(i, j) = A[i * n + j]
      TT_CUDA_CHECK(cudaMemsetAsync(acm, 0, (size_t)m * n * sizeof(double), s));
      TT_TRY(add_strided(s, acm, m, n, 1, m, R.a, n, 1));
      TT_TRY(qr_adjoint(s, m, n, acm, R.q, R.r, dOutk, p, 1, dF, dAc, sc, status));
      // back to row-major
      TT_CUDA_CHECK(cudaMemsetAsync(dA, 0, (size_t)m * n * sizeof(double), s));
      TT_TRY(add_strided(s, dA, m, n, n, 1, dAc, 1, m));
    } else {
      // u (m x p cm): tall u = Q U_R, wide u = U (the square factor is R_t^T, m x m)
      double* u = sc.take((size_t)m * p);
      double* P = sc.take((size_t)p * rn);
      double* G = sc.take((size_t)p * p);
      double* T = sc.take((size_t)p * n);
      double* X = sc.take((size_t)m * rn);
      double* H = sc.take((size_t)p * n);
      if (!u || !P || !G || !T || !X || !H) return fail(TT_ERR_WORKSPACE, "tt_round_backward: workspace too small");
      if (R.tall) TT_TRY(gemm64(s, m, p, p, 1.0, R.q, 1, m, R.u, 1, p, 0.0, u, 1, m));
      else TT_CUDA_CHECK(cudaMemcpyAsync(u, R.u, (size_t)m * p * sizeof(double), cudaMemcpyDeviceToDevice, s));
      // dF (rn x n rm) = g (rn x cols) next^T;  dC_rl[k+1] = F^T g (F rn x n rm)
      TT_TRY(gemm64(s, rn, n, cols, 1.0, g, cols, 1, R.next, 1, cols, 0.0, dF, n, 1));
      TT_TRY(gemm64(s, n, cols, rn, 1.0, R.f, 1, n, g, cols, 1, 0.0, dcrl[k + 1], cols, 1));
      // dB (m x rn, stored cm in X) = dout_k (m x rn rm) + A dF^T  (A m x n rm)
      TT_TRY(gemm64(s, m, rn, n, 1.0, R.a, n, 1, dF, 1, n, 0.0, X, 1, m));
      TT_TRY(add_strided(s, X, m, rn, 1, m, dOutk, rn, 1));
      // P = u^T dB (p x rn), G from P and sigma, T = u^T A (p x n)
      TT_TRY(gemm64(s, p, rn, m, 1.0, u, m, 1, X, 1, m, 0.0, P, 1, p));
      double s1 = 0.0;
      TT_CUDA_CHECK(cudaMemcpyAsync(&s1, R.sigma, sizeof(double), cudaMemcpyDeviceToHost, s));
      TT_CUDA_CHECK(cudaStreamSynchronize(s));
      svd_adj_g_kernel<<<blocks_for((int64_t)p * p), 256, 0, s>>>(P, p, rn, R.sigma, guard * s1 * s1, G);
      TT_LAUNCH_CHECK();
      TT_TRY(gemm64(s, p, n, m, 1.0, u, m, 1, R.a, n, 1, 0.0, T, 1, p));
      // dA (rm) = u (G T)
      TT_TRY(gemm64(s, p, n, p, 1.0, G, 1, p, T, 1, p, 0.0, H, 1, p));
      TT_TRY(gemm64(s, m, n, p, 1.0, u, 1, m, H, 1, p, 0.0, dA, n, 1));
      // + (dB - u P) S_r^{-2} T[:rn]
      TT_TRY(gemm64(s, m, rn, p, -1.0, u, 1, m, P, 1, p, 1.0, X, 1, m));
      scale_cols_inv2_kernel<<<blocks_for((int64_t)m * rn), 256, 0, s>>>(X, m, rn, R.sigma);
      TT_LAUNCH_CHECK();
      TT_TRY(gemm64(s, m, n, rn, 1.0, X, 1, m, T, 1, p, 1.0, dA, n, 1));
      // + B dF, B = u[:, :rn]
      TT_TRY(gemm64(s, m, n, rn, 1.0, u, 1, m, dF, n, 1, 1.0, dA, n, 1));
    }
    std::swap(g, g2);  // g <- dA: the cotangent of core k before the bond
    sc.off = mark;
  }
  // ---- 3. reverse of the right-to-left sweep; g is now the cotangent of the sweep's core 0,
  // i.e. of D_0 = x_0 R_1^T (rows x p row-major)
  double* dd = g;
  for (int k = 1; k < L; ++k) {
    const RoundRecord::RL& R = rec.rl[k];
    const int m = R.m, n = R.n, p = R.p, rows = R.rows_prev;
    const size_t mark = sc.off;
    double* dR = sc.take((size_t)p * n);
    double* ddt = sc.take((size_t)m * n);
    if (!dR || !ddt) return fail(TT_ERR_WORKSPACE, "tt_round_backward: workspace too small");
    // D_{k-1} (rows x p rm) = xprev (rows x n rm) R^T (R p x n cm): dx_{k-1} += dd R, dR = dd^T xprev
    TT_TRY(gemm64(s, rows, n, p, 1.0, dd, p, 1, R.r, 1, p, 1.0, static_cast<double*>(dx->cores[k - 1]), n, 1));
    TT_TRY(gemm64(s, p, n, rows, 1.0, dd, 1, p, R.xprev, n, 1, 0.0, dR, 1, p));
    // QR adjoint of dt (m x n cm) = q r; dq (m x p cm) is the output core's cotangent:
    // the core k is q^T row-major (p x m), so dq(i, j) = dcrl[k][j * m + i]
    TT_TRY(qr_adjoint(s, m, n, R.dt, R.q, R.r, dcrl[k], 1, m, dR, ddt, sc, status));
    // D_k (n x m rm) has the memory of dt (m x n cm): its cotangent is ddt as is
    TT_CUDA_CHECK(cudaMemcpyAsync(dd, ddt, (size_t)m * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    sc.off = mark;
  }
  {
    const size_t nl = (size_t)x->ranks[L - 1] * x->d[L - 1] * x->ranks[L];
    TT_TRY(add_strided(s, static_cast<double*>(dx->cores[L - 1]), (int)nl, 1, 1, 0, dd, 1, 0));
  }
  for (int k = 0; k < L; ++k) {
    const int64_t nk = x->ranks[k] * (int64_t)x->d[k] * x->ranks[k + 1];
    finite_kernel<<<blocks_for(nk), 256, 0, s>>>(static_cast<const double*>(dx->cores[k]), nk, status);
    TT_LAUNCH_CHECK();
  }
  unsigned st = 0;
  TT_CUDA_CHECK(cudaMemcpyAsync(&st, status, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  TT_CUDA_CHECK(cudaStreamSynchronize(s));
  if (st & ST_NONFINITE)
    return fail(TT_ERR_NUMERIC, "tt_round_backward: non-finite gradient (a right-to-left factor is singular: "
                                "x has bond ranks above the ranks of its unfoldings)");
  return TT_OK;
}

}  // namespace tt
