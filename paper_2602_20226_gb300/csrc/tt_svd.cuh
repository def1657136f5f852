// FP64 bond SVD (one-sided Jacobi) and truncation used by tt_round.
#pragma once

#include "tt_common.cuh"

namespace tt {

struct SvdWork {
  static constexpr int kMaxSweeps = 40;
  double* X = nullptr;  // p x n, column-major (X = R), ld ldx; rotated in place
  int ldx = 0;
  double* sigma = nullptr;  // [p] sorted descending
  int* perm = nullptr;      // [p] column of sigma_sorted[t]
  int* rank = nullptr;      // device int: truncated rank
  unsigned* bar = nullptr;  // [2] grid barrier state
  unsigned* rot = nullptr;  // [kMaxSweeps] rotations per sweep
  unsigned* status = nullptr;
  int* sweeps = nullptr;
  double* norm = nullptr;   // device double ||x||
  unsigned* epoch = nullptr;  // [p] per-column round counters (dataflow Jacobi); null: barrier per round
};

// One-sided Jacobi on the columns of X (nrow x ncol); the rotations are not kept.
// delta_scale > 0: pairs of columns that the truncation at delta = delta_scale * (*norm)
// discards in any case are skipped.
int jacobi_svd(cudaStream_t s, SvdWork& w, int nrow, int ncol, double tol, int max_sweeps,
               double delta_scale = 0.0);

// FP32 one-sided Jacobi, block round-robin in shared memory; the rotations are accumulated
// in V (V = I on entry is set here) unless V is null.  *w.sweeps
// receives the sweep count, or -1 if max_sweeps passed without convergence (no status
// flag is raised: the caller finishes the SVD in FP64 then).
size_t jacobi_block_smem(int nrow, int ncol);
int jacobi_block_f32(cudaStream_t s, SvdWork& w, float* X, int nrow, int ncol, int ldx, float* V, int ldv,
                     int max_sweeps);

// sigma, perm and the truncation rank with delta = delta_scale * (*norm); singular values
// below rel_floor * sigma_1 are dropped as well (0 in the FP64 form).
int svd_truncate(cudaStream_t s, SvdWork& w, int nrow, int ncol, double delta_scale,
                 int64_t max_rank, double rel_floor = 0.0);

// No-truncation certificate for the upper-triangular p x p factor R (FP64, ld ldr):
// *w.rank <- 1 if sigma_min(R) > max(1.01 delta, rel_floor ||R||_F), delta =
// delta_scale * (*w.norm), is proven, else 0.  The bound allows p*unit*||R||_F of error;
// unit = 2^-53, the certificate's own FP64 arithmetic, in both forms: the FP64 form's R
// is FP64, and the mixed form truncates on the singular values of its stored FP32 factor
// (copied exactly into R), so a certificate for that factor is what its SVD step would
// decide (rel_floor = the mixed form's 2^-22 floor).  Uses w.sigma as scratch.
int certify_full_rank(cudaStream_t s, SvdWork& w, const double* R, int p, int ldr, double delta_scale,
                      double unit, double rel_floor);

// ---- batched forms (one job per train of a batch, jobs in device memory)
struct SvdJob {
  double* X;        // n x n FP64 factor, column-major, ld ldx (rotated in place / W)
  int n, ldx;
  float* X32;       // mixed form: FP32 copy of the factor, rotated in place
  int ld32;
  double* sigma;
  int* perm;
  int* rank;        // truncation rank (or the certificate flag)
  unsigned* status;
  int* sweeps;
  const double* norm;
  int r;            // svd_left_batched: columns to gather into U (n x r)
  void* U;
  double dscale;    // the train's delta / ||x|| = eps / sqrt(L - 1)
};
// The batched SVD kernels take each job's delta from J.dscale * *J.norm, so trains of
// different lengths share one launch.
int certify_batched(cudaStream_t s, int nj, const SvdJob* d_jobs, int n_max, double unit, double rel_floor);
// Bond SVDs of a batch, one thread-block cluster of cs CTAs per job, all
// jobs of similar size: svd_cluster_size(n, fp64) picks cs (1 to 16) for bond rank n.
int svd_cluster_size(int n, bool fp64);
// skip: leave pairs of two negligible columns alone (each ||x||^2 < delta^2 / (2 n));
// false rotates every pair (the FP64 finish of the mixed form's FP32 sweeps)
int jacobi_f64_batched(cudaStream_t s, int nj, const SvdJob* d_jobs, int n_max, bool skip,
                       int max_sweeps, int cs);
// FP32 form: rotates J.X32 into W (rotations not accumulated); *sweeps = -1 when a job's
// FP32 sweeps did not settle (its caller finishes it in FP64).
int jacobi_f32_batched(cudaStream_t s, int nj, const SvdJob* d_jobs, int n_max, int max_sweeps, int cs);
int svd_truncate_batched(cudaStream_t s, int nj, const SvdJob* d_jobs, int n_max, int64_t max_rank,
                         double rel_floor);
template <typename TO>
int svd_left_batched(cudaStream_t s, int nj, const SvdJob* d_jobs, int64_t max_elems);
size_t jacobi_block_smem_gs(int gs, int nrow, int ncol);

// U (nrow x r, column-major) = X[:, perm[:r]] / sigma[:r]  (left singular vectors).
template <typename TO>
int svd_left_vectors(cudaStream_t s, const SvdWork& w, int nrow, int r, TO* U);

}  // namespace tt
