// FP64 bond SVD by one-sided Jacobi (Hestenes), truncation decision, gather.
//
// The rounding sweep needs the SVD of R (p x n, from the QR of a core).  We run
// one-sided Jacobi on the columns of X = R: plane rotations J make the columns of
// W = R J mutually orthogonal, so R = W J^T = U diag(sigma) V^T with sigma_j = ||W_j||
// and U = W diag(1/sigma).  The rotations are NOT accumulated: the truncated factors
// are formed from U alone,
//     C_k     <- Q U[:, perm[:r']]                  (orthonormal columns)
//     C_{k+1} <- (U[:, perm[:r']]^T R) C_{k+1}      (= (S V^T)[:r'] C_{k+1})
// so the kept part is an orthogonal projection of R whatever rounding the rotation
// sequence accumulated.  (Accumulating J over the ~p rotations per column per sweep
// leaves ||J^T J - I|| ~ 1e-12 at p = 320, which showed up as a 1e-12 error of
// the rounded train; U's orthogonality is set directly by the stopping test.)
//
// Parallel ordering: round-robin tournament over the p columns; every round's p/2
// rotations are independent.  One warp per column pair, CTAs synchronised between
// rounds by a bounded grid barrier inside a cooperative launch (a single CTA uses
// __syncthreads).  Rotation angle by Rutishauser's formulas.
#include "tt_svd.cuh"

#include <vector>

namespace tt {

namespace {

__device__ __forceinline__ bool sweep_barrier(unsigned* bar, unsigned* status) {
  if (gridDim.x == 1) {
    __syncthreads();
    return true;
  }
  return grid_barrier(bar, gridDim.x, status);
}

template <int NT>
__global__ void __launch_bounds__(NT) jacobi_kernel(double* X, int nrow, int ncol, int ldx,
                                                    double tol, int max_sweeps, unsigned* bar,
                                                    unsigned* rot, unsigned* status,
                                                    int* sweeps_out) {
  constexpr int WPB = NT / 32;
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * WPB + (threadIdx.x >> 5);
  const int GW = gridDim.x * WPB;
  const int N = ncol + (ncol & 1);
  const int npairs = N / 2;

  int sweep = 0;
  bool converged = false;
  for (; sweep < max_sweeps && !converged; ++sweep) {
    for (int rnd = 0; rnd < N - 1; ++rnd) {
      for (int q = gw; q < npairs; q += GW) {
        int a, b;
        if (q == 0) {
          a = rnd;
          b = N - 1;
        } else {
          a = (rnd + q) % (N - 1);
          b = (rnd - q + N - 1) % (N - 1);
        }
        if (a >= ncol || b >= ncol) continue;
        if (a > b) {
          const int t = a;
          a = b;
          b = t;
        }
        double* xa = X + (int64_t)a * ldx;
        double* xb = X + (int64_t)b * ldx;
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int i = lane; i < nrow; i += 32) {
          const double u = __ldcg(xa + i), v = __ldcg(xb + i);
          al = fma(u, u, al);
          be = fma(v, v, be);
          ga = fma(u, v, ga);
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (ga != 0.0 && fabs(ga) > tol * sqrt(al) * sqrt(be)) {
          const double zeta = (be - al) / (2.0 * ga);
          const double t = (fabs(zeta) > 1e150)
                               ? 0.5 / zeta
                               : copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double c = 1.0 / sqrt(1.0 + t * t);
          const double s = c * t;
          if (s == 0.0) continue;  // angle below resolution: nothing to rotate
          for (int i = lane; i < nrow; i += 32) {
            const double u = __ldcg(xa + i), v = __ldcg(xb + i);
            __stcg(xa + i, c * u - s * v);
            __stcg(xb + i, s * u + c * v);
          }
          if (lane == 0) atomicAdd(rot + sweep, 1u);
        }
      }
      if (!sweep_barrier(bar, status)) return;
    }
    converged = (*(volatile unsigned*)(rot + sweep) == 0u);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *sweeps_out = sweep;
    if (!converged) atomicOr(status, (unsigned)ST_NONCONVERGED);
  }
}

// sigma_j = ||X[:, j]||, sorted descending (stable), and the truncation rank:
// the smallest r >= 1 with sqrt(sum_{j >= r} sigma_j^2) <= delta, accumulated from
// the smallest singular value upwards, then capped at max_rank.
__global__ void __launch_bounds__(1024) svd_truncate_kernel(
    const double* X, int nrow, int ncol, int ldx, const double* norm, double delta_scale,
    long long max_rank, double* sig_sorted, int* perm, int* rank_out, unsigned* status) {
  extern __shared__ double sh[];
  double* sig = sh;
  double* srt = sh + ncol;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int c = warp; c < ncol; c += nw) {
    const double* col = X + (int64_t)c * ldx;
    double s = 0.0;
    for (int i = lane; i < nrow; i += 32) {
      const double v = __ldcg(col + i);
      s = fma(v, v, s);
    }
    s = warp_sum(s);
    if (lane == 0) sig[c] = sqrt(s);
  }
  __syncthreads();
  for (int j = tid; j < ncol; j += blockDim.x) {
    const double sj = sig[j];
    int r = 0;
    for (int q = 0; q < ncol; ++q) {
      const double sq = sig[q];
      r += (sq > sj) || (sq == sj && q < j);
    }
    perm[r] = j;
    srt[r] = sj;
    sig_sorted[r] = sj;
  }
  __syncthreads();
  if (tid == 0) {
    const double nrm = *norm;
    const double delta = delta_scale * nrm;
    bool finite = isfinite(nrm);
    double tail2 = 0.0;
    int r = ncol;
    for (int j = ncol - 1; j >= 1; --j) {
      const double t = fma(srt[j], srt[j], tail2);
      if (sqrt(t) <= delta) {
        tail2 = t;
        r = j;
      } else {
        break;
      }
    }
    for (int j = 0; j < ncol; ++j) finite = finite && isfinite(srt[j]);
    if (!finite) atomicOr(status, (unsigned)ST_NONFINITE);
    if (r > nrow) r = nrow;  // R has rank <= its row count
    if (r < 1) r = 1;
    if (max_rank > 0 && r > max_rank) r = (int)max_rank;
    *rank_out = r;
  }
}

// U[:, t] = X[:, perm[t]] / sigma_t  (nrow x r, column-major); zero column if sigma_t = 0
template <typename TO>
__global__ void svd_left_kernel(const double* X, int nrow, int ldx, const int* perm,
                                const double* sig_sorted, int r, TO* U) {
  const int64_t total = (int64_t)nrow * r;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % nrow), t = (int)(e / nrow);
    const double sg = sig_sorted[t];
    U[e] = (sg > 0.0) ? (TO)(__ldcg(X + i + (int64_t)perm[t] * ldx) / sg) : TO(0);
  }
}

struct CoopCfg {
  int dev = -1;
  int max_blocks = 0;
};

int coop_max_blocks(int threads) {
  static CoopCfg cfg;
  int dev = 0;
  TT_CUDA_CHECK(cudaGetDevice(&dev));
  if (cfg.dev != dev) {
    int occ = 0;
    TT_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, jacobi_kernel<64>, threads, 0));
    cfg.max_blocks = occ * num_sms();
    cfg.dev = dev;
  }
  return cfg.max_blocks;
}

}  // namespace

int jacobi_svd(cudaStream_t s, SvdWork& w, int nrow, int ncol, double tol, int max_sweeps) {
  if (ncol <= 0 || nrow <= 0) return TT_OK;
  if (max_sweeps > SvdWork::kMaxSweeps) max_sweeps = SvdWork::kMaxSweeps;
  TT_CUDA_CHECK(cudaMemsetAsync(w.bar, 0, 2 * sizeof(unsigned), s));
  TT_CUDA_CHECK(cudaMemsetAsync(w.rot, 0, SvdWork::kMaxSweeps * sizeof(unsigned), s));
  const int npairs = (ncol + 1) / 2;
  if (ncol <= 48) {
    jacobi_kernel<256><<<1, 256, 0, s>>>(w.X, nrow, ncol, w.ldx, tol, max_sweeps, w.bar, w.rot,
                                          w.status, w.sweeps);
    TT_LAUNCH_CHECK();
    return TT_OK;
  }
  constexpr int NT = 64;
  const int maxb = coop_max_blocks(NT);
  int blocks = (int)std::min<int64_t>(ceil_div(npairs, NT / 32), maxb);
  if (blocks < 1) blocks = 1;
  double* X = w.X;
  int ldx = w.ldx;
  unsigned *bar = w.bar, *rot = w.rot, *st = w.status;
  int* sw = w.sweeps;
  void* args[] = {&X, &nrow, &ncol, &ldx, &tol, &max_sweeps, &bar, &rot, &st, &sw};
  TT_CUDA_CHECK(cudaLaunchCooperativeKernel((const void*)jacobi_kernel<NT>, dim3(blocks), dim3(NT),
                                            args, 0, s));
  note_launch();
  return TT_OK;
}

int svd_truncate(cudaStream_t s, SvdWork& w, int nrow, int ncol, double delta_scale,
                 int64_t max_rank) {
  const size_t smem = 2 * (size_t)ncol * sizeof(double);
  if (smem > 200 * 1024) return fail(TT_ERR_UNSUPPORTED, "svd_truncate: bond rank too large");
  static int configured_dev = -1;
  int dev = 0;
  TT_CUDA_CHECK(cudaGetDevice(&dev));
  if (configured_dev != dev) {
    TT_CUDA_CHECK(cudaFuncSetAttribute(svd_truncate_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    configured_dev = dev;
  }
  svd_truncate_kernel<<<1, 1024, smem, s>>>(w.X, nrow, ncol, w.ldx, w.norm, delta_scale,
                                            (long long)max_rank, w.sigma, w.perm, w.rank, w.status);
  TT_LAUNCH_CHECK();
  return TT_OK;
}

template <typename TO>
int svd_left_vectors(cudaStream_t s, const SvdWork& w, int nrow, int r, TO* U) {
  const int64_t total = (int64_t)nrow * r;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(total, 256), 4096));
  svd_left_kernel<TO><<<blocks, 256, 0, s>>>(w.X, nrow, w.ldx, w.perm, w.sigma, r, U);
  TT_LAUNCH_CHECK();
  return TT_OK;
}

template int svd_left_vectors<double>(cudaStream_t, const SvdWork&, int, int, double*);
template int svd_left_vectors<float>(cudaStream_t, const SvdWork&, int, int, float*);

}  // namespace tt
