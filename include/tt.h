/*
 * libtt — quantics tensor-train arithmetic on sm_103a (C ABI).
 *
 * Every entry point is an operation of the trainsum paper (arXiv 2602.20226):
 *   tt_apply_mpo   'ij,j->i' of an MPO and a TT, core by core     Section 3.1, Eq. (quant_sum), Eq. (einsum)
 *   tt_hadamard    'i,i->i' of two TTs (element-wise product)      Section 3.1, Eq. (einsum)
 *   tt_round       normalisation centre to the left end, then a
 *                  truncated decomposition at each bond            Section 3.2 (decomposition algorithms);
 *                                                                  TensorTrain.truncate in Section 6
 *   tt_inner       'i,i->' (all indices contracted)                Section 3.1, Eq. (einsum)
 *   tt_eval        entries at index tuples (exact sampling)        Section 3.4; evaluate in Section 6
 * and the hand-written adjoint of each (the *_backward calls).
 *
 * Data layout (all row-major, all device memory unless stated):
 *   TT core k      G_k[r_{k-1}][d_k][r_k], r_0 = r_L = 1, site 1 = most significant digit
 *                  (Section 2, Eq. (quantization)).
 *   MPO core k     W_k[a_{k-1}][d_k (out i)][d_k (in j)][a_k].
 *   Bond flatten   a product bond is xi = mu * R_second + nu (first operand major),
 *                  the flatten xi = (mu, nu) after Eq. (einsum).
 *
 * Ownership: the caller allocates every buffer (device cores, device workspace,
 * host descriptor arrays) and keeps it alive until the stream work has finished.
 * The library never allocates or frees device memory.
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 * stream).  Calls enqueue work on that stream.  Calls that return a scalar or a
 * data-dependent rank to the host (tt_round, tt_inner) synchronise the stream.
 *
 * Errors: every call returns a tt_status.  Arguments are validated on the host
 * before anything is enqueued; on a validation error nothing is launched.
 * tt_last_error() returns a message for the last failing call of this thread.
 *
 * Threads: calls may come from several host threads at once, on any devices, as long as
 * they use different workspaces (and tt_inner_noalloc, whose scratch is shared, is not
 * overlapped).  The per-device launch settings the library caches on first use (SM count,
 * occupancy, shared-memory opt-ins) are kept in atomics.
 */
#ifndef LIBTT_TT_H
#define LIBTT_TT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TT_OK = 0,
  TT_ERR_ARG = 1,          /* NULL pointer or invalid scalar argument */
  TT_ERR_SHAPE = 2,        /* inconsistent lengths, modes or ranks */
  TT_ERR_DTYPE = 3,        /* unsupported or mismatched element type */
  TT_ERR_UNSUPPORTED = 4,  /* size beyond a documented limit */
  TT_ERR_WORKSPACE = 5,    /* workspace smaller than the *_workspace_size query */
  TT_ERR_CUDA = 6,         /* a CUDA runtime call failed */
  TT_ERR_NUMERIC = 7,      /* NaN/Inf met, or the Jacobi SVD hit its sweep cap */
  TT_ERR_TIMEOUT = 8       /* a bounded device-side wait expired */
} tt_status;

typedef enum { TT_F64 = 0, TT_F32 = 1 } tt_dtype;

/* Arithmetic form of tt_round.
 *   TT_PREC_FP64    everything in FP64 (the plain FP64 GPU form; TT_F64 cores).
 *   TT_PREC_MIXED   TT_F32 cores.  Every Householder panel is factored in FP64 and rounded
 *                   to FP32, with tau and the T factor recomputed in FP64 from the rounded
 *                   reflectors; the block-reflector updates keep W1 = V^T X and W2 = T^T W1
 *                   in FP64 and sum V W2 with exact products in float-float (compensated
 *                   FP32 arithmetic), rounding X once; the core GEMMs run on the tensor
 *                   cores in the sliced form of tt_gemm_f32_sliced (exact tensor-core sums)
 *                   where its tiles fill the GPU, compensated FP32 dot products below that;
 *                   a bond whose stored factor an FP64 certificate proves full rank skips
 *                   its SVD, the others get an FP64 preconditioning QR (of the factor's
 *                   transpose) and an FP32 one-sided Jacobi (the FP64 one above the FP32
 *                   kernel's shared-memory size); singular values, the truncation decision
 *                   and the norm in FP64. */
typedef enum { TT_PREC_FP64 = 0, TT_PREC_MIXED = 1 } tt_prec;

/* Size limits of the library. */
#define TT_MAX_SITES 128 /* L <= TT_MAX_SITES */
#define TT_MAX_MODE 16   /* d_k <= TT_MAX_MODE */

/* A tensor train.  Host-side descriptor of device cores.
 *   L      number of sites (1 <= L <= TT_MAX_SITES)
 *   dtype  tt_dtype of every core
 *   d      host [L], mode sizes d_k >= 1
 *   ranks  host [L+1], ranks[0] = ranks[L] = 1; output calls write it
 *   cores  host [L] array of device pointers; core k holds ranks[k]*d[k]*ranks[k+1]
 *          elements (for outputs of tt_round: room for the input's ranks). */
typedef struct {
  int32_t L;
  int32_t dtype;
  const int32_t* d;
  int64_t* ranks;
  void* const* cores;
} tt_train;

/* A matrix product operator with square cores W_k[a][d_k][d_k][a'].
 * Fields as in tt_train; ranks are the operator bonds a_k. */
typedef struct {
  int32_t L;
  int32_t dtype;
  const int32_t* d;
  const int64_t* ranks;
  void* const* cores;
} tt_mpo;

/* Message for the last failing call of the calling thread ("" if none). */
const char* tt_last_error(void);

/* Library version string. */
const char* tt_version(void);

/* y = W x ('ij,j->i', Section 3.1, Eq. (quant_sum) and Eq. (einsum)).
 *   Y_k[(a, r), i, (a', r')] = sum_j W_k[a, i, j, a'] G_k[r, j, r'],  xi = a * R_x + r.
 * y->ranks is written (ranks a_k * r_k); y->cores must hold those sizes.
 * W, x, y share dtype.  One launch for all sites.  Asynchronous. */
int tt_apply_mpo(const tt_mpo* W, const tt_train* x, tt_train* y, void* stream);

/* z = x (.) y ('i,i->i', Section 3.1, Eq. (einsum)).
 *   Z_k[(r, s), i, (r', s')] = X_k[r, i, r'] Y_k[s, i, s'].
 * z->ranks is written (ranks r_k * s_k).  Asynchronous. */
int tt_hadamard(const tt_train* x, const tt_train* y, tt_train* z, void* stream);

/* Device workspace (bytes) that tt_round needs for input x in form prec. */
size_t tt_round_workspace_size(const tt_train* x, int32_t prec);

/* out = round(x, eps, max_rank): TT rounding (Section 3.2).
 *   1. right-to-left sweep, k = L..2: LQ of C_k as r_{k-1} x (d_k r_k) by Householder
 *      QR of its transpose; C_k <- Q, C_{k-1} <- C_{k-1} L.  ||x|| = ||C_1||_F.
 *   2. left-to-right sweep, k = 1..L-1: QR of C_k as (r_{k-1} d_k) x r_k, SVD of R
 *      (one-sided Jacobi, FP64), r' = smallest r' >= 1 whose discarded singular
 *      values have 2-norm <= eps ||x|| / sqrt(L-1), capped at max_rank (<= 0: no cap);
 *      C_k <- Q U[:, :r'], C_{k+1} <- (S V^T)[:r'] C_{k+1}.
 * Guarantees ||x - out|| <= eps ||x|| when the cap does not bind.
 *   x      input TT (not modified); TT_F64 for TT_PREC_FP64, TT_F32 for TT_PREC_MIXED
 *   out    out->cores[k] must hold x's ranks[k]*d[k]*ranks[k+1] elements; the result
 *          is written compactly with its own ranks, which go to out->ranks (host).
 *   norm_out  host pointer or NULL; receives ||x|| (FP64)
 *   workspace/ws_bytes  device scratch of at least tt_round_workspace_size bytes.
 * Synchronises the stream (the truncated ranks are read back after every bond).
 * Returns TT_ERR_NUMERIC if a Jacobi SVD did not converge within its sweep cap
 * (the output is still written and still meets the error bound). */
int tt_round(const tt_train* x, double eps, int64_t max_rank, int32_t prec, tt_train* out,
             double* norm_out, void* workspace, size_t ws_bytes, void* stream);

/* Device workspace (bytes) that tt_round_backward needs for input x. */
size_t tt_round_backward_workspace_size(const tt_train* x);

/* Adjoint of tt_round in the FP64 form (Section 3.2's two sweeps, reversed):
 *   dx += d loss / dx, given dout = d loss / d out for out = tt_round(x, eps, max_rank,
 *   TT_PREC_FP64).
 * The forward rounding is run again (the same arithmetic as tt_round, so the same output
 * cores and gauge), recording its factors; then the left-to-right bonds are reversed (thin-QR
 * adjoint for the bonds the full-rank certificate kept, the adjoint of the leading left
 * singular vectors for the truncated ones, near-degenerate kept pairs guarded) and the
 * right-to-left steps (thin-QR adjoints).
 *   x      TT_F64 input of the rounding; dout TT_F64 with the ranks of out; dx TT_F64 with x's
 *          ranks, accumulated (+=).
 * The derivative exists where the truncation ranks are locally constant (a gap at every cut)
 * and every right-to-left factor has full rank, i.e. no bond rank of x exceeds the rank of
 * its unfolding; TT_ERR_NUMERIC (non-finite gradient) otherwise.  The loss should not depend
 * on the gauge of out's cores (e.g. a function of the represented tensor).  TT_ERR_SHAPE if
 * dout's ranks differ from round(x)'s.  Synchronises the stream. */
int tt_round_backward(const tt_train* x, double eps, int64_t max_rank, const tt_train* dout, tt_train* dx,
                      void* workspace, size_t ws_bytes, void* stream);

/* ---- batched apply + round over many independent trains ---- */

/* Device workspace (bytes) for tt_apply_round_batched: one rounding workspace per train
 * (sized for its apply output) plus the job arrays of the lock-step driver.  nstreams is
 * accepted for compatibility and does not change the size.  0 on invalid input. */
size_t tt_apply_round_batched_workspace_size(int32_t n, const tt_mpo* W, const tt_train* x,
                                             int32_t prec, int32_t nstreams);

/* For i < n: y[i] = W[i] x[i] (tt_apply_mpo), then out[i] = round(y[i], eps, max_rank)
 * (the rounding of tt_round in form prec; the same truncation rule per train, with
 * eps ||y[i]|| / sqrt(L_i - 1)).  Trains may differ in length, modes and ranks; all
 * must have the dtype of prec (TT_F64 / TT_PREC_FP64, TT_F32 / TT_PREC_MIXED).
 * The trains advance in lock-step: each step of the two sweeps is one launch per
 * operation over all trains that have that step (one job per train, own sizes), and
 * the host synchronises once per step for the truncation ranks.  The work runs on
 * streams[0]; streams[1..4] (when given) run the size classes of a step's bond SVDs side
 * by side (event fork / join on streams[0]).  The job descriptors are staged in one
 * pinned host buffer per process (allocated on first use, kept for reuse).
 *   y, out   caller-allocated outputs (y[i] sized for ranks a_k r_k; out[i] like
 *            tt_round's output); out[i].ranks receive the rounded ranks.
 *   workspace/ws_bytes  device scratch of tt_apply_round_batched_workspace_size bytes.
 * Returns when every train is done (stream synchronised); a failing train's status is
 * returned (TT_ERR_NUMERIC for a Jacobi sweep cap or non-finite values). */
int tt_apply_round_batched(int32_t n, const tt_mpo* W, const tt_train* x, tt_train* y, double eps,
                           int64_t max_rank, int32_t prec, tt_train* out, void* workspace,
                           size_t ws_bytes, void* const* streams, int32_t nstreams);

/* Device workspace (bytes) that tt_inner / tt_inner_backward need. */
size_t tt_inner_workspace_size(const tt_train* x, const tt_train* y);

/* <x, y> = E_L with E_0 = 1, E_k = sum_i X_k(i)^T E_{k-1} Y_k(i)  ('i,i->').
 * Environments are accumulated in FP64 for both dtypes.  *out (host) receives the
 * value; the call synchronises the stream. */
int tt_inner(const tt_train* x, const tt_train* y, double* out, void* workspace, size_t ws_bytes,
             void* stream);

/* <x, y> exactly as tt_inner, for callers that cannot supply or allocate device
 * memory: plain C programs embedding the library without a device allocator of their
 * own, and latency-critical loops under a fixed memory budget, where cudaMalloc /
 * cudaFree would synchronise the device.  This call takes no workspace and allocates
 * nothing.  (The paper has no counterpart; it is an interface convenience.)
 *   Scratch: a fixed 4 MiB device array inside the library, held by every GPU that
 *   loads the library until the process exits.  Trains whose tt_inner_workspace_size
 *   exceeds 4 MiB are rejected with TT_ERR_UNSUPPORTED before anything is launched.
 *   Set-up: the first call on each device looks up the array's device address (with
 *   that device current); make that first call before any stream capture.  The address
 *   is kept for the life of the process: after cudaDeviceReset (or anything else that
 *   destroys the device's primary context) later calls on that device are invalid.
 *   Sharing: all calls on a device use the same array and it keeps the last call's
 *   contents, so calls that overlap on the GPU (other streams, other threads) race;
 *   serialise them.  Synchronises the stream like tt_inner. */
int tt_inner_noalloc(const tt_train* x, const tt_train* y, double* out, void* stream);

/* values[s] = G_1[:, i_1^s, :] ... G_L[:, i_L^s, :]  (exact evaluation).
 *   digits  device uint8 [n][L], digit k of sample s at digits[s*L + k] (< d_k)
 *   values  device [n], x's dtype.  Asynchronous. */
int tt_eval(const tt_train* x, const uint8_t* digits, int64_t n, void* values, void* stream);

/* ---- adjoints: gradients are ACCUMULATED (+=) into caller-initialised cores ---- */

/* dG_k[r, j, r'] += sum_{a, a', i} W_k[a, i, j, a'] dY_k[(a, r), i, (a', r')]
 * dW_k[a, i, j, a'] += sum_{r, r'} G_k[r, j, r'] dY_k[(a, r), i, (a', r')]   (dW may be NULL).
 * dy has y's shape (ranks a_k r_k).  Asynchronous. */
int tt_apply_mpo_backward(const tt_mpo* W, const tt_train* x, const tt_train* dy, tt_mpo* dW,
                          tt_train* dx, void* stream);

/* dX_k[r, i, r'] += sum_{s, s'} dZ_k[(r, s), i, (r', s')] Y_k[s, i, s'], and dY likewise
 * (either gradient may be NULL).  Asynchronous. */
int tt_hadamard_backward(const tt_train* x, const tt_train* y, const tt_train* dz, tt_train* dx,
                         tt_train* dy, void* stream);

/* dX_k(i) += dout E^L_{k-1} Y_k(i) (E^R_k)^T,  dY_k(i) += dout (E^L_{k-1})^T X_k(i) E^R_k,
 * with left environments E^L and right environments E^R (E^R_L = 1,
 * E^R_{k-1} = sum_i X_k(i) E^R_k Y_k(i)^T).  Either gradient may be NULL.
 * Environments in FP64.  Workspace: tt_inner_workspace_size.  Asynchronous. */
int tt_inner_backward(const tt_train* x, const tt_train* y, double dout, tt_train* dx,
                      tt_train* dy, void* workspace, size_t ws_bytes, void* stream);

/* Device workspace (bytes) that tt_eval_backward needs for n samples.  Samples are
 * processed in chunks whose prefix and suffix states take at most 1 GiB (at most 65536
 * samples), so the size stops growing beyond one chunk. */
size_t tt_eval_backward_workspace_size(const tt_train* x, int64_t n);

/* dG_k[:, i, :] += sum_{s : i_k^s = i} dvalues_s prefix_s^T suffix_s, where
 * prefix_s = G_1[:, i_1^s, :] ... G_{k-1}[:, i_{k-1}^s, :] and suffix_s is the
 * product of the cores right of k (paper Sec. 3.4, evaluation; the gradient is linear in
 * dvalues).  Prefixes and suffixes are formed and stored in x's dtype; the sums over
 * samples run in x's dtype over slices of at most 2048 samples and are accumulated across
 * slices in FP64.  Samples whose digit at a site is out of range add nothing there.
 * dvalues: device [n], x's dtype.  Cores of dx that are NULL are skipped.  Asynchronous. */
int tt_eval_backward(const tt_train* x, const uint8_t* digits, int64_t n, const void* dvalues,
                     tt_train* dx, void* workspace, size_t ws_bytes, void* stream);

/* ---- diagnostics ---- */

/* Exercises the library's bounded device-side wait (the wait of the dataflow Jacobi SVDs)
 * on a flag that nothing sets: the wait gives up after poll_limit polls, raises the timeout
 * bit of a device status word and the kernel returns; the call then returns TT_ERR_TIMEOUT
 * and the CUDA context stays usable.  scratch: caller-allocated device memory of at least
 * 12 bytes (zeroed by the call).  poll_limit in [1, 2^24] (the library's own limit), else
 * TT_ERR_ARG.  Synchronises the stream.  No counterpart in the paper (failure handling). */
int tt_debug_wait_expiry(int64_t poll_limit, void* scratch, void* stream);

/* Number of CUDA kernels this library has launched in this process so far (all
 * threads, all devices).  A caller reads it before and after a region of work to
 * count the launches inside it. */
uint64_t tt_launch_count(void);

/* Event profiler of tt_round.  tt_profile_enable(1) clears the counters and turns it
 * on (0 turns it off).  While on, tt_round brackets each phase with a pair of CUDA
 * events on its own stream and accumulates, per class, the elapsed time, the nominal
 * flops of the phase and the number of phases:
 *   class 0  Jacobi SVD launches (12 p^3 flops each for a p x p factor)
 *   class 1  Householder QR with thin Q (4 m n^2 - 4 n^3 / 3)
 *   class 2  the GEMMs that form the new cores (2 m n k)
 *   class 3  full-rank certificates (p^3 / 3 flops: the inverse of a p x p triangle)
 * tt_profile_read returns TT_ERR_ARG for an unknown class. */
void tt_profile_enable(int32_t on);
int tt_profile_read(int32_t cls, double* ms, double* nominal_flops, uint64_t* count);

/* Executed work of a profiler class since tt_profile_enable(1), where it differs from the
 * nominal count: for class 0 the Jacobi work that actually ran - per sweep of a p x p factor
 * the three dot products of every pair of columns (6 p flops a pair), plus 6 p flops for each
 * rotation applied (FP64 form; the mixed form's FP32 sweeps count 12 p flops a pair), plus the
 * QR of R^T that preconditions FP64 factors (4 p^3 / 3); bonds whose SVD the full-rank
 * certificate skipped contribute nothing.  The other classes equal their nominal flops.
 * TT_ERR_ARG for an unknown class. */
int tt_profile_read_executed(int32_t cls, double* executed_flops);

/* C = alpha A B + beta C in FP32 on the tensor cores: TF32 with a 3-term hi/lo split
 * (A_hi B_hi + A_hi B_lo + A_lo B_hi, FP32 accumulation).  Not on the rounding path: the
 * tensor cores round each accumulation toward zero, a bias the mixed form cannot afford
 * (tt_gemm_f32_sliced is the form it uses).  No counterpart in the paper.
 * Element (m, k) of A is A[m*sam + k*sak], (k, n) of B is B[k*sbk + n*sbn], (m, n) of
 * C is C[m*scm + n*scn] (device pointers; any strides).  beta = 0 never reads C.
 * Asynchronous. */
int tt_gemm_f32(int32_t M, int32_t N, int32_t K, double alpha, const float* A, int64_t sam,
                int64_t sak, const float* B, int64_t sbk, int64_t sbn, double beta, float* C,
                int64_t scm, int64_t scn, void* stream);

/* C = alpha A B + beta C in FP32 on the tensor cores in the sliced form, the GEMM of the
 * mixed form of tt_apply_round_batched (and of tt_round where its tiles fill the GPU).
 * Per 32-wide block of K,
 * each row of A and each column of B is scaled by its own power of two and cut into
 * three signed integer slices rounded to nearest (h1 + 2^-9 h2 + 2^-18 h3, |h1| <= 512,
 * |h2|, |h3| <= 256); six TF32 tcgen05 MMAs per K step form three level sums of slice
 * products, integers below 2^24 and therefore exact whatever the tensor core's rounding;
 * the levels are scaled and added in float-float.  Error per element <= 2^-20 sum over
 * 32-wide K blocks of max|a| max|b| (the dropped h2 h3, h3 h2, h3 h3 terms and the last
 * slice's rounding; zero-mean), plus the final rounding to FP32.  Rows or
 * columns whose block maximum is below 2^-118 count as zero in that block.  No
 * counterpart in the paper (Ozaki-type splitting).  Arguments as tt_gemm_f32; K = 0
 * scales C by beta.  Asynchronous. */
int tt_gemm_f32_sliced(int32_t M, int32_t N, int32_t K, double alpha, const float* A, int64_t sam,
                       int64_t sak, const float* B, int64_t sbk, int64_t sbn, double beta, float* C,
                       int64_t scm, int64_t scn, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* LIBTT_TT_H */
