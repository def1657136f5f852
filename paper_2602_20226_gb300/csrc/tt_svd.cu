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

// Sum of (a, b, c) over a warp with 6 FP64 additions per lane instead of 15: the first two
// butterfly levels halve the number of values each lane carries ((a, b, c, 0) -> two -> one),
// the last three sum the one left.  On return the lane holds the total of value
// (lane >> 3) & 3 of (a, b, c, 0): lanes 0-7 a, 8-15 b, 16-23 c.
__device__ __forceinline__ double warp_sum3_split(double a, double b, double c, int lane) {
  const bool hi16 = lane & 16;
  double k0 = hi16 ? c : a, k1 = hi16 ? 0.0 : b;
  const double s0 = hi16 ? a : c, s1 = hi16 ? b : 0.0;
  k0 += __shfl_xor_sync(0xffffffffu, s0, 16);
  k1 += __shfl_xor_sync(0xffffffffu, s1, 16);
  const bool hi8 = lane & 8;
  double k = hi8 ? k1 : k0;
  k += __shfl_xor_sync(0xffffffffu, hi8 ? k0 : k1, 8);
  k += __shfl_xor_sync(0xffffffffu, k, 4);
  k += __shfl_xor_sync(0xffffffffu, k, 2);
  k += __shfl_xor_sync(0xffffffffu, k, 1);
  return k;
}

// Columns of up to 32 * TPL rows are held in registers for the whole pair update
// (all loads issued at once, one store pass); TPL = 0 streams longer columns.
template <int TPL>
__device__ __forceinline__ bool rotate_pair(double* __restrict__ xa, double* __restrict__ xb,
                                            int nrow, int lane, double tol, double negl) {
  double al = 0.0, be = 0.0, ga = 0.0;
  double ra[TPL > 0 ? TPL : 1], rb[TPL > 0 ? TPL : 1];
  if (TPL > 0) {
    // chunks wholly beyond nrow are skipped by a warp-uniform test (an FP64 instruction with
    // every lane predicated off still takes its 16 clocks of the SM's FP64 pipe)
#pragma unroll
    for (int t = 0; t < TPL; ++t) {
      ra[t] = rb[t] = 0.0;
      if (32 * t < nrow) {
        const int i = lane + 32 * t;
        if (i < nrow) {
          ra[t] = __ldcg(xa + i);
          rb[t] = __ldcg(xb + i);
        }
      }
    }
#pragma unroll
    for (int t = 0; t < TPL; ++t) {
      if (32 * t < nrow) {
        al = fma(ra[t], ra[t], al);
        be = fma(rb[t], rb[t], be);
        ga = fma(ra[t], rb[t], ga);
      }
    }
  } else {
    for (int i = lane; i < nrow; i += 32) {
      const double u = __ldcg(xa + i), v = __ldcg(xb + i);
      al = fma(u, u, al);
      be = fma(v, v, be);
      ga = fma(u, v, ga);
    }
  }
  const double v = warp_sum3_split(al, be, ga, lane);
  al = __shfl_sync(0xffffffffu, v, 0);
  be = __shfl_sync(0xffffffffu, v, 8);
  ga = __shfl_sync(0xffffffffu, v, 16);
  if (al < negl && be < negl) return false;  // both columns are truncated whatever the angle
  if (!(ga != 0.0 && fabs(ga) > tol * sqrt(al) * sqrt(be))) return false;
  const double zeta = (be - al) / (2.0 * ga);
  const double t = (fabs(zeta) > 1e150) ? 0.5 / zeta
                                        : copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
  const double c = 1.0 / sqrt(1.0 + t * t);
  const double s = c * t;
  if (s == 0.0) return false;  // angle below resolution: nothing to rotate
  if (TPL > 0) {
#pragma unroll
    for (int q = 0; q < TPL; ++q) {
      if (32 * q < nrow) {
        const int i = lane + 32 * q;
        if (i < nrow) {
          __stcg(xa + i, c * ra[q] - s * rb[q]);
          __stcg(xb + i, s * ra[q] + c * rb[q]);
        }
      }
    }
  } else {
    for (int i = lane; i < nrow; i += 32) {
      const double u = __ldcg(xa + i), v = __ldcg(xb + i);
      __stcg(xa + i, c * u - s * v);
      __stcg(xb + i, s * u + c * v);
    }
  }
  return true;
}

// Epoch handshake of the dataflow ordering: column c has been through epoch[c] rounds.
// Lane 0 waits (bounded) until column c has finished round t-1, i.e. epoch[c] >= t.
__device__ __forceinline__ bool wait_column(const unsigned* epoch, int c, unsigned t, unsigned* status) {
  return bounded_wait_ge(epoch + c, t, status);
}

// FLOW = false: a grid barrier after every round (p - 1 per sweep).
// FLOW = true (dataflow ordering): each column carries an epoch counter; the warp that
// takes pair (a, b) in round t waits only until both columns have left round t - 1 (an
// acquire load of their counters), rotates them and releases both counters to t + 1.
// In the round-robin ordering every column is in exactly one pair per round, so the
// dependencies of a pair are the two pairs that last held its columns; warps run ahead
// as far as their inputs allow and a grid barrier is needed only once per sweep, for
// the convergence test.  All CTAs are co-resident (cooperative launch) and every warp
// takes its rounds in order, so the waits cannot form a cycle; each wait is bounded.
template <int NT, int TPL, bool FLOW>
__global__ void __launch_bounds__(NT) jacobi_kernel(double* X, int nrow, int ncol, int ldx,
                                                    double tol, double negl_scale, const double* norm,
                                                    int max_sweeps, unsigned* bar, unsigned* rot,
                                                    unsigned* status, int* sweeps_out, unsigned* epoch) {
  constexpr int WPB = NT / 32;
  const double nl = negl_scale > 0.0 ? negl_scale * __ldcg(norm) : 0.0;
  const double negl = nl * nl;
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * WPB + (threadIdx.x >> 5);
  const int GW = gridDim.x * WPB;
  const int N = ncol + (ncol & 1);
  const int npairs = N / 2;

  int sweep = 0;
  bool converged = false;
  bool ok = true;
  unsigned t = 0;  // rounds completed before the current one (dataflow epoch)
  for (; sweep < max_sweeps && !converged; ++sweep) {
    for (int rnd = 0; rnd < N - 1; ++rnd, ++t) {
      for (int q = gw; ok && q < npairs; q += GW) {
        int a, b;
        if (q == 0) {
          a = rnd;
          b = N - 1;
        } else {
          a = (rnd + q) % (N - 1);
          b = (rnd - q + N - 1) % (N - 1);
        }
        if (a > b) {
          const int tmp = a;
          a = b;
          b = tmp;
        }
        // a < b, so only b can be the padding column N - 1 (odd ncol)
        const bool real_b = b < ncol;
        if (FLOW) {
          int good = 1;
          if (lane == 0) good = wait_column(epoch, a, t, status) && (!real_b || wait_column(epoch, b, t, status));
          good = __shfl_sync(0xffffffffu, good, 0);
          if (!good) {
            ok = false;
            break;
          }
        }
        if (real_b && rotate_pair<TPL>(X + (int64_t)a * ldx, X + (int64_t)b * ldx, nrow, lane, tol, negl) &&
            lane == 0)
          atomicAdd(rot + sweep, 1u);
        if (FLOW) {
          __syncwarp();
          if (lane == 0) {
            __threadfence();
            st_release_u32(epoch + a, t + 1);
            if (real_b) st_release_u32(epoch + b, t + 1);
          }
        }
      }
      if (!FLOW && !sweep_barrier(bar, status)) return;
    }
    if (FLOW && !sweep_barrier(bar, status)) return;  // also ends a CTA whose wait expired
    converged = (*(volatile unsigned*)(rot + sweep) == 0u);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *sweeps_out = sweep;
    if (!converged) atomicOr(status, (unsigned)ST_NONCONVERGED);
  }
}

// The rotation of one-sided Jacobi for a pair with squared norms al, be and product ga, or
// false if the pair is left alone.  tan(theta) is the smaller root of t^2 + 2 zeta t - 1 = 0,
// zeta = (be - al) / (2 ga), written as t = sgn(d) 2 ga / (|d| + sqrt(d^2 + 4 ga^2)) with
// d = be - al: one square root, one division and one reciprocal square root on the
// dependent chain (the zeta form has three divisions and three square roots).  The sums are
// first scaled by a power of two (exact), so d^2 + 4 ga^2 can neither overflow nor underflow,
// and the acceptance test |ga| > tol sqrt(al be) is taken as ga^2 > tol^2 al be on them.
__device__ __forceinline__ bool jacobi_rotation(double al, double be, double ga, double tol, double negl, double& c,
                                                double& sn) {
  if ((al < negl && be < negl) || ga == 0.0) return false;
  const int e = ilogb(fmax(al, be));
  al = scalbn(al, -e);
  be = scalbn(be, -e);
  ga = scalbn(ga, -e);
  if (!(ga * ga > (tol * tol) * (al * be))) return false;
  const double d = be - al;
  const double h = sqrt(fma(d, d, 4.0 * ga * ga));
  const double t = copysign(1.0, d) * (2.0 * ga) / (fabs(d) + h);
  c = rsqrt(fma(t, t, 1.0));
  sn = c * t;
  return sn != 0.0;
}

// FP64 one-sided Jacobi of a factor of at most 64 x 64 in one CTA of 8 warps, round-robin
// ordering, the factor held in shared memory for the whole run.  Each round runs in three
// phases: every warp forms the three dot products of its (up to four) pairs, rows over
// lanes, keeping the columns in registers; warp 0 derives the rotations of all the round's
// pairs at once, one pair per lane (jacobi_rotation), so the square roots and divisions are
// issued once per round rather than once per pair - at 2 FP64 lanes per clock per SM they
// dominated small factors; the warps apply them.
constexpr int kSmallJacobi = 64;

__global__ void __launch_bounds__(256) jacobi_small_kernel(double* X, int nrow, int ncol, int ldx, double tol,
                                                           double negl_scale, const double* norm, int max_sweeps,
                                                           unsigned* rot, unsigned* status, int* sweeps_out) {
  constexpr int TPL = kSmallJacobi / 32, PPW = kSmallJacobi / 2 / 8;
  __shared__ double s_abg[32][3];
  __shared__ double s_cs[32][2];
  __shared__ int s_do[32];
  extern __shared__ double Xs[];  // the factor, column-major, ld nrow: it stays on chip
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int e = threadIdx.x; e < nrow * ncol; e += blockDim.x) {
    const int i = e % nrow, col = e / nrow;
    Xs[e] = X[i + (int64_t)col * ldx];
  }
  __syncthreads();
  const double nl = negl_scale > 0.0 ? negl_scale * __ldcg(norm) : 0.0;
  const double negl = nl * nl;
  const int N = ncol + (ncol & 1), npairs = N / 2;
  int sweep = 0;
  bool converged = false;
  for (; sweep < max_sweeps && !converged; ++sweep) {
    unsigned nrot = 0;  // warp 0, lane 0
    for (int rnd = 0; rnd < N - 1; ++rnd) {
      double ra[PPW][TPL], rb[PPW][TPL];
      // ---- phase A: dot products of this warp's pairs
#pragma unroll
      for (int j = 0; j < PPW; ++j) {
        const int q = warp + 8 * j;
        int a = 0, b = 0;
        if (q < npairs) {
          a = q == 0 ? rnd : (rnd + q) % (N - 1);
          b = q == 0 ? N - 1 : (rnd - q + N - 1) % (N - 1);
          if (a > b) {
            const int t = a;
            a = b;
            b = t;
          }
        }
        double al = 0.0, be = 0.0, ga = 0.0;
#pragma unroll
        for (int u = 0; u < TPL; ++u) {
          ra[j][u] = rb[j][u] = 0.0;
          if (q < npairs && b < ncol && 32 * u < nrow) {
            const int i = lane + 32 * u;
            if (i < nrow) {
              ra[j][u] = Xs[i + a * nrow];
              rb[j][u] = Xs[i + b * nrow];
            }
            al = fma(ra[j][u], ra[j][u], al);
            be = fma(rb[j][u], rb[j][u], be);
            ga = fma(ra[j][u], rb[j][u], ga);
          }
        }
        if (q < npairs) {
          const double v = warp_sum3_split(al, be, ga, lane);
          if ((lane & 7) == 0 && lane < 24) s_abg[q][lane >> 3] = v;
        }
      }
      __syncthreads();
      // ---- phase B: the rotations, one pair per lane of warp 0
      if (warp == 0) {
        int doit = 0;
        double c = 1.0, sn = 0.0;
        if (lane < npairs) {
          int a = lane == 0 ? rnd : (rnd + lane) % (N - 1);
          int b = lane == 0 ? N - 1 : (rnd - lane + N - 1) % (N - 1);
          if (a > b) b = a;  // only b can be the padding column N - 1
          if (b < ncol) doit = jacobi_rotation(s_abg[lane][0], s_abg[lane][1], s_abg[lane][2], tol, negl, c, sn);
          if (!doit) {
            c = 1.0;
            sn = 0.0;
          }
          s_cs[lane][0] = c;
          s_cs[lane][1] = sn;
          s_do[lane] = doit;
        }
        nrot += __popc(__ballot_sync(0xffffffffu, doit));
      }
      __syncthreads();
      // ---- phase C: apply
#pragma unroll
      for (int j = 0; j < PPW; ++j) {
        const int q = warp + 8 * j;
        if (q < npairs && s_do[q]) {
          int a = q == 0 ? rnd : (rnd + q) % (N - 1);
          int b = q == 0 ? N - 1 : (rnd - q + N - 1) % (N - 1);
          if (a > b) {
            const int t = a;
            a = b;
            b = t;
          }
          const double c = s_cs[q][0], sn = s_cs[q][1];
#pragma unroll
          for (int u = 0; u < TPL; ++u) {
            if (32 * u < nrow) {
              const int i = lane + 32 * u;
              if (i < nrow) {
                Xs[i + a * nrow] = c * ra[j][u] - sn * rb[j][u];
                Xs[i + b * nrow] = sn * ra[j][u] + c * rb[j][u];
              }
            }
          }
        }
      }
      __syncthreads();
    }
    __shared__ unsigned s_nrot;
    if (threadIdx.x == 0) {
      s_nrot = nrot;
      if (nrot) atomicAdd(rot + sweep, nrot);
    }
    __syncthreads();
    converged = s_nrot == 0u;
    __syncthreads();  // s_nrot is read before the next sweep overwrites it
  }
  for (int e = threadIdx.x; e < nrow * ncol; e += blockDim.x) {
    const int i = e % nrow, col = e / nrow;
    X[i + (int64_t)col * ldx] = Xs[e];
  }
  if (threadIdx.x == 0) {
    *sweeps_out = sweep;
    if (!converged) atomicOr(status, (unsigned)ST_NONCONVERGED);
  }
}

// The same FP64 Jacobi with one CTA of WPP warps per pair: the rows of the pair are split
// over the warps (shorter dependent FMA chains, WPP times the warps per SM), the partial
// sums are combined in shared memory in a fixed order, and one thread derives the rotation
// for the whole CTA.  GB300's FP64 rate is 2 lanes per clock per SM, so every FP64
// instruction a warp issues holds the SM's FP64 pipe for 16 clocks: the divisions and square
// roots of the rotation (about 60 FP64 instructions) are issued once, not by every warp; the
// warp sums take 6 additions per lane (warp_sum3_split); register chunks wholly beyond a
// warp's rows are skipped by a warp-uniform test instead of being issued with every lane
// predicated off.  Dataflow ordering between pairs as in jacobi_kernel.
template <int WPP, int TPL>
__global__ void __launch_bounds__(32 * WPP) jacobi_wpp_kernel(double* X, int nrow, int ncol, int ldx, double tol,
                                                             double negl_scale, const double* norm, int max_sweeps,
                                                             unsigned* bar, unsigned* rot, unsigned* status,
                                                             int* sweeps_out, unsigned* epoch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double nl = negl_scale > 0.0 ? negl_scale * __ldcg(norm) : 0.0;
  const double negl = nl * nl;
  const int N = ncol + (ncol & 1), npairs = N / 2;
  const int rows = (nrow + WPP - 1) / WPP;  // rows of one warp
  const int i_lo = warp * rows, i_hi = min(nrow, i_lo + rows);
  __shared__ double red[WPP][3];
  __shared__ double s_cs[2];
  __shared__ int s_ok, s_doit;
  int sweep = 0;
  bool converged = false;
  unsigned t = 0;
  for (; sweep < max_sweeps && !converged; ++sweep) {
    for (int rnd = 0; rnd < N - 1; ++rnd, ++t) {
      for (int q = blockIdx.x; q < npairs; q += gridDim.x) {
        int a, b;
        if (q == 0) {
          a = rnd;
          b = N - 1;
        } else {
          a = (rnd + q) % (N - 1);
          b = (rnd - q + N - 1) % (N - 1);
        }
        if (a > b) {
          const int tmp = a;
          a = b;
          b = tmp;
        }
        const bool real_b = b < ncol;
        if (threadIdx.x == 0) s_ok = wait_column(epoch, a, t, status) && (!real_b || wait_column(epoch, b, t, status));
        __syncthreads();
        if (!s_ok) {
          // leave through the sweep barrier, which sees ST_TIMEOUT
          q = npairs;
          rnd = N;
          break;
        }
        double* xa = X + (int64_t)a * ldx;
        double* xb = X + (int64_t)b * ldx;
        if (real_b) {
          double ra[TPL], rb[TPL];
          double al = 0.0, be = 0.0, ga = 0.0;
#pragma unroll
          for (int u = 0; u < TPL; ++u) {
            ra[u] = rb[u] = 0.0;
            if (i_lo + 32 * u < i_hi) {  // warp-uniform
              const int i = i_lo + lane + 32 * u;
              if (i < i_hi) {
                ra[u] = __ldcg(xa + i);
                rb[u] = __ldcg(xb + i);
              }
            }
          }
#pragma unroll
          for (int u = 0; u < TPL; ++u) {
            if (i_lo + 32 * u < i_hi) {
              al = fma(ra[u], ra[u], al);
              be = fma(rb[u], rb[u], be);
              ga = fma(ra[u], rb[u], ga);
            }
          }
          const double v = warp_sum3_split(al, be, ga, lane);
          if ((lane & 7) == 0 && lane < 24) red[warp][lane >> 3] = v;
          __syncthreads();
          if (threadIdx.x == 0) {
            al = be = ga = 0.0;
#pragma unroll
            for (int w = 0; w < WPP; ++w) {
              al += red[w][0];
              be += red[w][1];
              ga += red[w][2];
            }
            double c = 1.0, sn = 0.0;
            const bool doit = jacobi_rotation(al, be, ga, tol, negl, c, sn);
            s_cs[0] = c;
            s_cs[1] = sn;
            s_doit = doit;
            if (doit) atomicAdd(rot + sweep, 1u);
          }
          __syncthreads();
          if (s_doit) {
            const double c = s_cs[0], sn = s_cs[1];
#pragma unroll
            for (int u = 0; u < TPL; ++u) {
              if (i_lo + 32 * u < i_hi) {
                const int i = i_lo + lane + 32 * u;
                if (i < i_hi) {
                  __stcg(xa + i, c * ra[u] - sn * rb[u]);
                  __stcg(xb + i, sn * ra[u] + c * rb[u]);
                }
              }
            }
          }
        }
        // every warp's stores (and reads of red / s_cs) precede the release: the CTA barrier
        // orders them before thread 0's st.release.gpu, and a release is cumulative, so a CTA
        // that acquires the epoch sees the rotated columns (no separate fence.sc needed)
        __syncthreads();
        if (threadIdx.x == 0) {
          st_release_u32(epoch + a, t + 1);
          if (real_b) st_release_u32(epoch + b, t + 1);
        }
      }
    }
    if (!sweep_barrier(bar, status)) return;
    converged = (*(volatile unsigned*)(rot + sweep) == 0u);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *sweeps_out = sweep;
    if (!converged) atomicOr(status, (unsigned)ST_NONCONVERGED);
  }
}

// FP32 one-sided Jacobi with accumulated rotations, organised as a block round-robin:
// the columns are cut into groups of 16; in each outer round a CTA takes one pair of
// groups (32 columns of X and of V) into shared memory and rotates the 256 pairs across
// the two groups (16 inner rounds of 16 rotations, one warp per pair, __syncthreads between
// inner rounds; in a sweep's first outer round also the pairs inside each group), then
// writes them back.  Group pairs follow the round-robin order,
// so a grid barrier is needed only between outer rounds: 2G - 1 per sweep for G
// groups instead of p - 1.  The mixed form uses it as the fast part of its bond SVD.
// Global -> shared copy of the C2 columns listed in cols (n values each, column c of
// src at src + cols[c] * ld; -1 = zero column), U independent loads in flight per
// thread so the copy costs a few L2 latencies, not one per element.
template <int U>
__device__ __forceinline__ void load_cols(float* __restrict__ dst, const float* __restrict__ src,
                                          const int* cols, int C2, int n, int ld) {
  const int total = C2 * n;
  for (int base = threadIdx.x; base < total; base += blockDim.x * U) {
    float v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = base + u * blockDim.x;
      v[u] = 0.f;
      if (e < total) {
        const int c = e / n;
        if (cols[c] >= 0) v[u] = __ldcg(src + (e - c * n) + (int64_t)cols[c] * ld);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = base + u * blockDim.x;
      if (e < total) dst[e] = v[u];
    }
  }
}

__device__ __forceinline__ void store_cols(const float* __restrict__ srcs, float* __restrict__ dst,
                                           const int* cols, int C2, int n, int ld) {
  const int total = C2 * n;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int c = e / n;
    if (cols[c] >= 0) __stcg(dst + (e - c * n) + (int64_t)cols[c] * ld, srcs[e]);
  }
}

// One FP32 Jacobi rotation of the shared-memory columns (xa, xb) of length nrow, applied
// to (va, vb) of length ncol as well; the columns are read in chunks of 32 * TPL values
// held in registers (one chunk: read once, rotated from registers).
template <int TPL>
__device__ __forceinline__ bool rotate_pair_f32(float* xa, float* xb, float* va, float* vb, int nrow,
                                                int ncol, int lane, float tol, float negl) {
  constexpr int CH = 32 * TPL;
  float ra[TPL], rb[TPL];
  float al = 0.f, be = 0.f, ga = 0.f;
  for (int i0 = 0; i0 < nrow; i0 += CH) {
#pragma unroll
    for (int t = 0; t < TPL; ++t) {
      const int i = i0 + lane + 32 * t;
      ra[t] = i < nrow ? xa[i] : 0.f;
      rb[t] = i < nrow ? xb[i] : 0.f;
    }
#pragma unroll
    for (int t = 0; t < TPL; ++t) {
      al = fmaf(ra[t], ra[t], al);
      be = fmaf(rb[t], rb[t], be);
      ga = fmaf(ra[t], rb[t], ga);
    }
  }
  al = warp_sum(al);
  be = warp_sum(be);
  ga = warp_sum(ga);
  if (al < negl && be < negl) return false;  // two noise-level columns: both are dropped
  if (!(ga != 0.f && fabsf(ga) > tol * sqrtf(al) * sqrtf(be))) return false;
  const float zeta = (be - al) / (2.f * ga);
  const float tn = (fabsf(zeta) > 1e18f) ? 0.5f / zeta
                                         : copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
  const float c = 1.f / sqrtf(1.f + tn * tn);
  const float s = c * tn;
  if (s == 0.f) return false;
  for (int i0 = 0; i0 < nrow; i0 += CH) {
    if (nrow > CH) {  // several chunks: the registers hold the last one, reload
#pragma unroll
      for (int t = 0; t < TPL; ++t) {
        const int i = i0 + lane + 32 * t;
        ra[t] = i < nrow ? xa[i] : 0.f;
        rb[t] = i < nrow ? xb[i] : 0.f;
      }
    }
#pragma unroll
    for (int t = 0; t < TPL; ++t) {
      const int i = i0 + lane + 32 * t;
      if (i < nrow) {
        xa[i] = c * ra[t] - s * rb[t];
        xb[i] = s * ra[t] + c * rb[t];
      }
    }
  }
  for (int i0 = 0; i0 < ncol; i0 += CH) {
#pragma unroll
    for (int t = 0; t < TPL; ++t) {
      const int i = i0 + lane + 32 * t;
      ra[t] = i < ncol ? va[i] : 0.f;
      rb[t] = i < ncol ? vb[i] : 0.f;
    }
#pragma unroll
    for (int t = 0; t < TPL; ++t) {
      const int i = i0 + lane + 32 * t;
      if (i < ncol) {
        va[i] = c * ra[t] - s * rb[t];
        vb[i] = s * ra[t] + c * rb[t];
      }
    }
  }
  return true;
}

// GS columns per group, one warp per pair of the 2 GS columns in shared memory.
// With gepoch (one counter per group) the outer rounds follow the same dataflow rule as
// jacobi_kernel: a CTA waits only for its two groups to leave the previous outer round,
// and the grid barrier runs once per sweep.
template <int GS, int TPL>
__global__ void __launch_bounds__(32 * GS) jacobi_block_f32_kernel(float* X, int nrow, int ncol, int ldx,
                                                                   float* V, int ldv, float tol,
                                                                   int max_sweeps, unsigned* bar,
                                                                   unsigned* rot, unsigned* status,
                                                                   int* sweeps_out, unsigned* gepoch,
                                                                   float negl_scale, const double* norm) {
  constexpr int kJbGroup = GS;
  const float nl = negl_scale > 0.f ? negl_scale * (float)__ldcg(norm) : 0.f;
  const float negl = nl * nl;
  extern __shared__ float jsm[];
  constexpr int C2 = 2 * kJbGroup;
  float* Xs = jsm;                           // C2 columns x nrow
  float* Vs = jsm + (size_t)C2 * nrow;       // C2 columns x ncol
  __shared__ int cols[C2];
  __shared__ unsigned s_rot;
  __shared__ int s_ok;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int G = (ncol + kJbGroup - 1) / kJbGroup;
  const int NG = G + (G & 1);
  const bool flow = gepoch != nullptr;
  int sweep = 0;
  bool converged = false;
  unsigned t = 0;  // outer rounds completed before the current one
  for (; sweep < max_sweeps && !converged; ++sweep) {
    for (int r = 0; r < NG - 1; ++r, ++t) {
      for (int q = blockIdx.x; q < NG / 2; q += gridDim.x) {
        int ga, gb;
        if (q == 0) {
          ga = r;
          gb = NG - 1;
        } else {
          ga = (r + q) % (NG - 1);
          gb = (r - q + NG - 1) % (NG - 1);
        }
        if (flow) {
          if (tid == 0)
            s_ok = (ga >= G || wait_column(gepoch, ga, t, status)) && (gb >= G || wait_column(gepoch, gb, t, status));
          __syncthreads();
          if (!s_ok) break;  // a wait expired: leave through the sweep barrier
        }
        if (tid < C2) {
          const int g = tid < kJbGroup ? ga : gb;
          const int c = g * kJbGroup + (tid % kJbGroup);
          cols[tid] = (g < G && c < ncol) ? c : -1;
        }
        if (tid == 0) s_rot = 0;
        __syncthreads();
        load_cols<8>(Xs, X, cols, C2, nrow, ldx);
        if (V) load_cols<8>(Vs, V, cols, C2, ncol, ldv);
        __syncthreads();
        // Each pair of columns once per sweep: the pairs inside each group in the sweep's first
        // outer round (every group takes part in it once; the two groups' round-robins side by
        // side, GS - 1 rounds of GS / 2 + GS / 2 pairs), and the GS x GS pairs across the two
        // groups in every outer round (GS rounds of GS disjoint pairs, slot w of the first group
        // with slot (w + ir) mod GS of the second)
        unsigned local = 0;
        if (r == 0) {
          constexpr int H = kJbGroup / 2;
          const int wg = warp % H, base = warp < H ? 0 : kJbGroup;
          for (int ir = 0; ir < kJbGroup - 1; ++ir) {
            int a, b;
            if (wg == 0) {
              a = ir;
              b = kJbGroup - 1;
            } else {
              a = (ir + wg) % (kJbGroup - 1);
              b = (ir - wg + kJbGroup - 1) % (kJbGroup - 1);
            }
            a += base;
            b += base;
            if (cols[a] >= 0 && cols[b] >= 0 &&
                rotate_pair_f32<TPL>(Xs + (size_t)a * nrow, Xs + (size_t)b * nrow, Vs + (size_t)a * ncol,
                                     Vs + (size_t)b * ncol, nrow, V ? ncol : 0, lane, tol, negl))
              ++local;
            __syncthreads();
          }
        }
        for (int ir = 0; ir < kJbGroup; ++ir) {
          const int a = warp, b = kJbGroup + (warp + ir) % kJbGroup;
          if (cols[a] >= 0 && cols[b] >= 0 &&
              rotate_pair_f32<TPL>(Xs + (size_t)a * nrow, Xs + (size_t)b * nrow, Vs + (size_t)a * ncol,
                                   Vs + (size_t)b * ncol, nrow, V ? ncol : 0, lane, tol, negl))
            ++local;
          __syncthreads();
        }
        if (lane == 0 && local) atomicAdd(&s_rot, local);
        store_cols(Xs, X, cols, C2, nrow, ldx);
        if (V) store_cols(Vs, V, cols, C2, ncol, ldv);
        __syncthreads();
        if (tid == 0 && s_rot) atomicAdd(rot + sweep, s_rot);
        if (flow && tid == 0) {
          __threadfence();
          if (ga < G) st_release_u32(gepoch + ga, t + 1);
          if (gb < G) st_release_u32(gepoch + gb, t + 1);
        }
      }
      if (flow && (*(volatile unsigned*)status & ST_TIMEOUT)) break;
      if (!flow && !sweep_barrier(bar, status)) return;
    }
    if (flow && !sweep_barrier(bar, status)) return;
    converged = (*(volatile unsigned*)(rot + sweep) == 0u);
  }
  // the caller decides what a cap means here: -1 reports it (no status flag)
  if (blockIdx.x == 0 && threadIdx.x == 0) *sweeps_out = converged ? sweep : -1;
}

__global__ void identity_f32_kernel(float* V, int n, int ldv) {
  const int64_t total = (int64_t)n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), c = (int)(e / n);
    V[i + (int64_t)c * ldv] = (i == c) ? 1.f : 0.f;
  }
}

// sigma_j = ||X[:, j]||, sorted descending (stable), and the truncation rank:
// the smallest r >= 1 with sqrt(sum_{j >= r} sigma_j^2) <= delta, accumulated from
// the smallest singular value upwards, then capped at max_rank.
__device__ __forceinline__ void svd_truncate_body(
    const double* X, int nrow, int ncol, int ldx, const double* norm, double delta_scale,
    long long max_rank, double rel_floor, double* sig_sorted, int* perm, int* rank_out,
    unsigned* status) {
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
  // rank by counting under a total order: NaN sorts last (key -inf) and ties go by index, so
  // the ranks form a permutation whatever the values (perm indexes columns later; a NaN
  // compared false both ways and left duplicate ranks and unset entries)
  for (int j = tid; j < ncol; j += blockDim.x) {
    const double sj = sig[j];
    const double kj = isnan(sj) ? -INFINITY : sj;
    int r = 0;
    for (int q = 0; q < ncol; ++q) {
      const double sq = sig[q];
      const double kq = isnan(sq) ? -INFINITY : sq;
      r += (kq > kj) || (kq == kj && q < j);
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
    // sqrt(t) <= delta decided without the square root away from the threshold: with
    // d2 = delta^2 rounded, t <= d2 (1 - 2^-48) implies sqrt(t) < delta (1 - 2^-50) and
    // t >= d2 (1 + 2^-48) implies sqrt(t) > delta (1 + 2^-50), beyond the rounding of the
    // square root either way; in between the square root is taken as before
    // (delta^2 outside the normal range, where the relative margins do not hold: always
    // the square root)
    const double d2 = delta * delta;
    const bool margins = d2 >= 0x1p-1000 && d2 <= 0x1p+1000;
    const double d2_lo = margins ? d2 * (1.0 - 0x1p-48) : -1.0, d2_hi = margins ? d2 * (1.0 + 0x1p-48) : INFINITY;
    for (int j = ncol - 1; j >= 1; --j) {
      const double t = fma(srt[j], srt[j], tail2);
      const bool keep_tail = t <= d2_lo ? true : (t >= d2_hi ? false : sqrt(t) <= delta);
      if (keep_tail) {
        tail2 = t;
        r = j;
      } else {
        break;
      }
    }
    for (int j = 0; j < ncol; ++j) finite = finite && isfinite(srt[j]);
    if (!finite) atomicOr(status, (unsigned)ST_NONFINITE);
    if (r > nrow) r = nrow;  // R has rank <= its row count
    // singular values below the resolution of the arithmetic that produced the factor
    // (rel_floor * sigma_1) are not kept, whatever delta allows
    while (r > 1 && srt[r - 1] < rel_floor * srt[0]) --r;
    if (r < 1) r = 1;
    if (max_rank > 0 && r > max_rank) r = (int)max_rank;
    *rank_out = r;
  }
}

__global__ void __launch_bounds__(1024) svd_truncate_kernel(
    const double* X, int nrow, int ncol, int ldx, const double* norm, double delta_scale,
    long long max_rank, double rel_floor, double* sig_sorted, int* perm, int* rank_out,
    unsigned* status) {
  svd_truncate_body(X, nrow, ncol, ldx, norm, delta_scale, max_rank, rel_floor, sig_sorted, perm, rank_out,
                    status);
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
    const int c = perm[t];  // a column of the square factor; out of range only by a bug: zero
    U[e] = (sg > 0.0 && (unsigned)c < (unsigned)nrow) ? (TO)(__ldcg(X + i + (int64_t)c * ldx) / sg) : TO(0);
  }
}

// No-truncation certificate for an upper-triangular R (p x p, column-major, FP64):
// sigma_min(R) >= 1 / ||R^{-1}||_F, and ||R^{-1}||_F comes from p independent
// back substitutions (one warp per column of R^{-1}).  The computed inverse is that
// of R + dR with |dR| <= p u |R|, so the certificate subtracts p u ||R||_F.  If
// sigma_min > delta, no singular value can be dropped (the smallest tail already
// exceeds delta) and the bond keeps its full rank.
__device__ __forceinline__ void rinv_colnorm_body(const double* R, int p, int ldr, double* colsq, int bx) {
  const int lane = threadIdx.x & 31;
  const int j = bx * 8 + (threadIdx.x >> 5);
  if (j >= p) return;
  // z = R^{-1} e_j: z_j = 1/R_jj, z_i = -(sum_{l=i+1..j} R_il z_l) / R_ii for i < j,
  // kept in this warp's slice of shared memory.
  extern __shared__ double zbuf[];  // 8 warps x p
  double* z = zbuf + (size_t)(threadIdx.x >> 5) * p;
  const double rjj = R[j + (int64_t)j * ldr];
  if (lane == 0) z[j] = 1.0 / rjj;
  __syncwarp();
  double nrm2 = (lane == 0) ? z[j] * z[j] : 0.0;
  for (int i = j - 1; i >= 0; --i) {
    double acc = 0.0;
    for (int l = i + 1 + lane; l <= j; l += 32) acc = fma(R[i + (int64_t)l * ldr], z[l], acc);
    acc = warp_sum(acc);
    const double zi = -acc / R[i + (int64_t)i * ldr];
    if (lane == 0) z[i] = zi;
    nrm2 = fma(zi, zi, nrm2);
    __syncwarp();
  }
  if (lane == 0) colsq[j] = nrm2;
}

// The same column norms, column-oriented: one warp per column j forms z = R^{-1} e_j by
//   for i = j .. 0:  z_i = b_i / R_ii;  b_k -= z_i R_ki  (k < i)
// with the right-hand side b in registers (b_k in lane k % 32, slot k / 32), so a step is
// one broadcast, one multiply and one FMA per slot - no warp reduction and no division
// on the critical path (the row-oriented form above needs both, and reads a row of the
// column-major R per step).  The CTA's warps share 32-column blocks of R (with the
// inverses of their diagonal) staged in shared memory.  p <= 32 KS.
constexpr int kRinvWarps = 4;

template <int KS>
__device__ __forceinline__ void rinv_colnorm_cols_body(const double* __restrict__ R, int p, int ldr,
                                                       double* __restrict__ colsq, int bx) {
  extern __shared__ double rs[];  // rows [0, c0 + 32) x 32 columns (ld = rows), then 32 inverse diagonals
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = bx * kRinvWarps + warp;
  const int jmax = min(p - 1, bx * kRinvWarps + kRinvWarps - 1);
  double b[KS];
#pragma unroll
  for (int q = 0; q < KS; ++q) b[q] = (32 * q + lane == j) ? 1.0 : 0.0;
  double nrm2 = 0.0;
#pragma unroll
  for (int B = KS - 1; B >= 0; --B) {
    if (32 * B > jmax) continue;  // CTA-uniform
    const int c0 = 32 * B, rows = min(p, c0 + 32), nc = min(32, p - c0);
    double* dinv = rs + (size_t)rows * 32;
    __syncthreads();  // the previous block is consumed
    for (int e = threadIdx.x; e < rows * nc; e += blockDim.x) {
      const int r = e % rows, cc = e / rows;
      rs[r + cc * rows] = __ldg(R + r + (int64_t)(c0 + cc) * ldr);
    }
    if (threadIdx.x < nc) dinv[threadIdx.x] = 1.0 / __ldg(R + (c0 + threadIdx.x) + (int64_t)(c0 + threadIdx.x) * ldr);
    __syncthreads();
    if (j < p) {
      const int top = min(31, j - c0);  // steps i = c0 + ii, ii = top .. 0 (i <= j)
      for (int ii = top; ii >= 0; --ii) {
        const double zi = __shfl_sync(0xffffffffu, b[B], ii) * dinv[ii];
        nrm2 = fma(zi, zi, nrm2);
        const double* col = rs + ii * rows;  // column c0 + ii of R, rows [0, c0 + 32)
#pragma unroll
        for (int q = 0; q < B; ++q) b[q] = fma(-zi, col[32 * q + lane], b[q]);
        if (lane < ii) b[B] = fma(-zi, col[c0 + lane], b[B]);
      }
    }
  }
  if (j < p && lane == 0) colsq[j] = nrm2;
}

template <int KS>
__global__ void __launch_bounds__(32 * kRinvWarps) rinv_colnorm_cols_kernel(const double* __restrict__ R, int p,
                                                                            int ldr, double* __restrict__ colsq) {
  rinv_colnorm_cols_body<KS>(R, p, ldr, colsq, blockIdx.x);
}

__global__ void __launch_bounds__(256) rinv_colnorm_kernel(const double* R, int p, int ldr,
                                                           double* colsq) {
  rinv_colnorm_body(R, p, ldr, colsq, blockIdx.x);
}

// flag = 1 if 1/||R^{-1}||_F - p u ||R||_F > max(1.01 delta, rel_floor ||R||_F) (certified
// full rank: sigma_min(R) exceeds both the truncation threshold and the relative floor
// below which the mixed form drops singular values), else 0.  u is the unit roundoff of
// the FP64 arithmetic that forms R^{-1} here.
__device__ __forceinline__ void certify_body(const double* R, int p, int ldr, const double* colsq,
                                             const double* norm, double delta_scale, double unit,
                                             double rel_floor, int* flag) {
  __shared__ double scratch[32];
  double inv2 = 0.0, r2 = 0.0;
  for (int j = threadIdx.x; j < p; j += blockDim.x) inv2 += colsq[j];
  for (int64_t e = threadIdx.x; e < (int64_t)p * p; e += blockDim.x) {
    const int i = (int)(e % p), c = (int)(e / p);
    if (i <= c) {
      const double v = R[i + (int64_t)c * ldr];
      r2 = fma(v, v, r2);
    }
  }
  inv2 = block_sum(inv2, scratch);
  r2 = block_sum(r2, scratch);
  if (threadIdx.x == 0) {
    const double delta = delta_scale * (*norm);
    const double lower = (isfinite(inv2) && inv2 > 0.0) ? 1.0 / sqrt(inv2) : 0.0;
    const double slack = (double)p * unit * sqrt(r2);
    *flag = (lower - slack > fmax(1.01 * delta, rel_floor * sqrt(r2))) ? 1 : 0;
  }
}

__global__ void __launch_bounds__(1024) certify_kernel(const double* R, int p, int ldr,
                                                       const double* colsq, const double* norm,
                                                       double delta_scale, double unit, double rel_floor,
                                                       int* flag) {
  certify_body(R, p, ldr, colsq, norm, delta_scale, unit, rel_floor, flag);
}

// ------------------------------------------------------------------ batched forms
// One job per train of a batch; every kernel below takes the job from its block index.

__global__ void __launch_bounds__(256) rinv_colnorm_batched_kernel(const SvdJob* __restrict__ jobs) {
  const SvdJob& J = jobs[blockIdx.y];
  if ((int)blockIdx.x * 8 >= J.n) return;
  rinv_colnorm_body(J.X, J.n, J.ldx, J.sigma, blockIdx.x);
}

// column-oriented form for the batch (bond ranks <= 32 KS): grid (ceil(n_max / 4), jobs)
template <int KS>
__global__ void __launch_bounds__(32 * kRinvWarps) rinv_colnorm_cols_batched_kernel(const SvdJob* __restrict__ jobs) {
  const SvdJob& J = jobs[blockIdx.y];
  if ((int)blockIdx.x * kRinvWarps >= J.n) return;  // the whole CTA leaves together
  rinv_colnorm_cols_body<KS>(J.X, J.n, J.ldx, J.sigma, blockIdx.x);
}

__global__ void __launch_bounds__(1024) certify_batched_kernel(const SvdJob* __restrict__ jobs, double unit,
                                                               double rel_floor) {
  const SvdJob& J = jobs[blockIdx.x];
  certify_body(J.X, J.n, J.ldx, J.sigma, J.norm, J.dscale, unit, rel_floor, J.rank);
}

__global__ void __launch_bounds__(1024) svd_truncate_batched_kernel(const SvdJob* __restrict__ jobs,
                                                                    long long max_rank, double rel_floor) {
  const SvdJob& J = jobs[blockIdx.x];
  svd_truncate_body(J.X, J.n, J.n, J.ldx, J.norm, J.dscale, max_rank, rel_floor, J.sigma, J.perm, J.rank,
                    J.status);
}

// Cluster forms: one thread-block cluster of CS CTAs per job (clusters are co-scheduled,
// so the per-job barriers are hardware cluster barriers).  CTA `rank` of a cluster takes
// every CS-th pair (FP64) or group pair (FP32) of a round; the columns stay in global
// memory (read and written through L2) and the cluster barrier after each round orders
// those accesses between the CTAs.  The sweep's rotation count is summed over the
// cluster through distributed shared memory.
__device__ __forceinline__ unsigned cluster_sum_u32(unsigned* slot, int cs, unsigned* bcast) {
  // *slot: this CTA's count (already final); returns the cluster total in every thread
  cluster_sync_all();
  if (threadIdx.x == 0) {
    unsigned t = 0;
    const unsigned a = (unsigned)__cvta_generic_to_shared(slot);
    for (int r = 0; r < cs; ++r) {
      unsigned ra, v;
      asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(r));
      asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(ra) : "memory");
      t += v;
    }
    *bcast = t;
  }
  cluster_sync_all();  // every CTA has read every slot before any resets its own
  return *bcast;
}

template <int NT, int TPL, int CS>
__global__ void __launch_bounds__(NT) jacobi_f64_cluster_kernel(const SvdJob* __restrict__ jobs, int skip,
                                                                int max_sweeps) {
  const int rank = (int)(blockIdx.x % CS);
  const SvdJob& J = jobs[blockIdx.x / CS];
  const int ncol = J.n, nrow = J.n;
  if (ncol <= 0) return;  // the whole cluster leaves together
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gw = rank * NW + warp, GW = CS * NW;
  const double tol = sqrt((double)ncol) * 2.220446049250313e-16;
  const double nl = (skip && J.dscale > 0.0) ? J.dscale * __ldcg(J.norm) / sqrt(2.0 * ncol) : 0.0;
  const double negl = nl * nl;
  const int N = ncol + (ncol & 1), npairs = N / 2;
  __shared__ unsigned s_rot, s_tot;
  int sweep = 0;
  bool converged = false;
  for (; sweep < max_sweeps && !converged; ++sweep) {
    if (threadIdx.x == 0) s_rot = 0;
    __syncthreads();
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
        if (a > b) {
          const int t = a;
          a = b;
          b = t;
        }
        if (b < ncol && rotate_pair<TPL>(J.X + (int64_t)a * J.ldx, J.X + (int64_t)b * J.ldx, nrow, lane, tol, negl) &&
            lane == 0)
          atomicAdd(&s_rot, 1u);
      }
      __syncthreads();
      cluster_sync_all();
    }
    converged = cluster_sum_u32(&s_rot, CS, &s_tot) == 0u;
  }
  if (rank == 0 && threadIdx.x == 0) {
    *J.sweeps = sweep;
    if (!converged) atomicOr(J.status, (unsigned)ST_NONCONVERGED);
  }
}

// FP32 rotation of the global columns (xa, xb) (length n) in chunks of 32 * TPL values held
// in registers (loads of a chunk issued together).
template <int TPL>
__device__ __forceinline__ bool rotate_pair_f32_global(float* __restrict__ xa, float* __restrict__ xb, int n,
                                                       int lane, float tol, float negl) {
  constexpr int CH = 32 * TPL;
  float ra[TPL], rb[TPL];
  float al = 0.f, be = 0.f, ga = 0.f;
  for (int i0 = 0; i0 < n; i0 += CH) {
#pragma unroll
    for (int t = 0; t < TPL; ++t) {
      const int i = i0 + lane + 32 * t;
      ra[t] = i < n ? __ldcg(xa + i) : 0.f;
      rb[t] = i < n ? __ldcg(xb + i) : 0.f;
    }
#pragma unroll
    for (int t = 0; t < TPL; ++t) {
      al = fmaf(ra[t], ra[t], al);
      be = fmaf(rb[t], rb[t], be);
      ga = fmaf(ra[t], rb[t], ga);
    }
  }
  al = warp_sum(al);
  be = warp_sum(be);
  ga = warp_sum(ga);
  if (al < negl && be < negl) return false;
  if (!(ga != 0.f && fabsf(ga) > tol * sqrtf(al) * sqrtf(be))) return false;
  const float zeta = (be - al) / (2.f * ga);
  const float tn = (fabsf(zeta) > 1e18f) ? 0.5f / zeta
                                         : copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
  const float c = 1.f / sqrtf(1.f + tn * tn);
  const float s = c * tn;
  if (s == 0.f) return false;
  for (int i0 = 0; i0 < n; i0 += CH) {
    if (n > CH) {
#pragma unroll
      for (int t = 0; t < TPL; ++t) {
        const int i = i0 + lane + 32 * t;
        ra[t] = i < n ? __ldcg(xa + i) : 0.f;
        rb[t] = i < n ? __ldcg(xb + i) : 0.f;
      }
    }
#pragma unroll
    for (int t = 0; t < TPL; ++t) {
      const int i = i0 + lane + 32 * t;
      if (i < n) {
        __stcg(xa + i, c * ra[t] - s * rb[t]);
        __stcg(xb + i, s * ra[t] + c * rb[t]);
      }
    }
  }
  return true;
}

// FP32 one-sided Jacobi (rotations not accumulated), plain round-robin ordering as the
// FP64 cluster kernel: the CS x NT / 32 warps of a job's cluster take the pairs of a
// round, one cluster barrier per round.  J.X32 ends with W = X J (sigma_j = ||W_j||).
template <int NT, int TPL, int CS>
__global__ void __launch_bounds__(NT) jacobi_f32rr_cluster_kernel(const SvdJob* __restrict__ jobs,
                                                                  int max_sweeps) {
  const int rank = (int)(blockIdx.x % CS);
  const SvdJob& J = jobs[blockIdx.x / CS];
  const int n = J.n;
  if (n <= 0) return;
  constexpr int NW = NT / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int gw = rank * NW + warp, GW = CS * NW;
  float* X = J.X32;
  const int ld = J.ld32;
  const float tol = 8.f * sqrtf((float)n) * 5.9604645e-8f;
  const float nl = (float)(__ldcg(J.norm) / (double)(1 << 22) / sqrt(2.0 * n));
  const float negl = nl * nl;
  const int N = n + (n & 1), npairs = N / 2;
  __shared__ unsigned s_rot, s_tot;
  if (tid == 0) s_rot = 0;
  __syncthreads();
  cluster_sync_all();
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
        if (a > b) {
          const int t = a;
          a = b;
          b = t;
        }
        if (b < n && rotate_pair_f32_global<TPL>(X + (int64_t)a * ld, X + (int64_t)b * ld, n, lane, tol, negl) &&
            lane == 0)
          atomicAdd(&s_rot, 1u);
      }
      __syncthreads();
      cluster_sync_all();
    }
    converged = cluster_sum_u32(&s_rot, CS, &s_tot) == 0u;
    if (tid == 0) s_rot = 0;
    __syncthreads();
  }
  if (rank == 0 && tid == 0) *J.sweeps = converged ? sweep : -1;
}

template <typename TO>
__global__ void svd_left_batched_kernel(const SvdJob* __restrict__ jobs) {
  const SvdJob& J = jobs[blockIdx.y];
  const int r = J.r, nrow = J.n;
  TO* U = static_cast<TO*>(J.U);
  const int64_t total = (int64_t)nrow * r;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % nrow), t = (int)(e / nrow);
    const double sg = J.sigma[t];
    const int c = J.perm[t];
    U[e] = (sg > 0.0 && (unsigned)c < (unsigned)nrow) ? (TO)(__ldcg(J.X + i + (int64_t)c * J.ldx) / sg) : TO(0);
  }
}

}  // namespace

template <int TPL>
int launch_wpp(cudaStream_t s, SvdWork& w, int nrow, int ncol, double tol, double negl_scale, int max_sweeps) {
  constexpr int WPP = 4, NT = 32 * WPP;
  static std::atomic<int> cfg_dev{-1}, cfg_blocks{0};  // blocks stored before the device tag
  int dev = 0;
  TT_CUDA_CHECK(cudaGetDevice(&dev));
  if (cfg_dev != dev) {
    int occ = 0;
    TT_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, jacobi_wpp_kernel<WPP, TPL>, NT, 0));
    cfg_blocks = occ * num_sms();
    cfg_dev = dev;
  }
  const int npairs = (ncol + 1) / 2;
  int blocks = std::min(npairs, cfg_blocks.load());
  if (blocks < 1) blocks = 1;
  TT_CUDA_CHECK(cudaMemsetAsync(w.epoch, 0, (size_t)ncol * sizeof(unsigned), s));
  double* X = w.X;
  int ldx = w.ldx;
  const double* nrm = w.norm;
  unsigned *bar = w.bar, *rot = w.rot, *st = w.status, *ep = w.epoch;
  int* sw = w.sweeps;
  void* args[] = {&X, &nrow, &ncol, &ldx, &tol, &negl_scale, &nrm, &max_sweeps, &bar, &rot, &st, &sw, &ep};
  TT_CUDA_CHECK(cudaLaunchCooperativeKernel((const void*)jacobi_wpp_kernel<WPP, TPL>, dim3(blocks), dim3(NT), args,
                                            0, s));
  note_launch();
  return TT_OK;
}

int launch_jacobi_wpp(cudaStream_t s, SvdWork& w, int nrow, int ncol, double tol, double negl_scale,
                      int max_sweeps) {
  // rows per warp = nrow / 4, in registers: 32 TPL >= that
  if (nrow <= 128) return launch_wpp<1>(s, w, nrow, ncol, tol, negl_scale, max_sweeps);
  if (nrow <= 256) return launch_wpp<2>(s, w, nrow, ncol, tol, negl_scale, max_sweeps);
  return launch_wpp<4>(s, w, nrow, ncol, tol, negl_scale, max_sweeps);
}

template <int NT, int TPL>
int launch_jacobi(cudaStream_t s, SvdWork& w, int nrow, int ncol, double tol, double negl_scale,
                  int max_sweeps) {
  const int npairs = (ncol + 1) / 2;
  if (ncol <= kSmallJacobi && nrow <= kSmallJacobi) {
    jacobi_small_kernel<<<1, 256, (size_t)nrow * ncol * sizeof(double), s>>>(w.X, nrow, ncol, w.ldx, tol, negl_scale,
                                                                            w.norm, max_sweeps, w.rot, w.status,
                                                                            w.sweeps);
    TT_LAUNCH_CHECK();
    return TT_OK;
  }
  if (ncol <= 48) {
    jacobi_kernel<256, TPL, false><<<1, 256, 0, s>>>(w.X, nrow, ncol, w.ldx, tol, negl_scale, w.norm,
                                                      max_sweeps, w.bar, w.rot, w.status, w.sweeps, nullptr);
    TT_LAUNCH_CHECK();
    return TT_OK;
  }
  // the dataflow ordering needs one epoch counter per column (SvdWork::epoch); with it,
  // one CTA of four warps per pair (rows split) when each warp gets at most 128 rows
  if (w.epoch != nullptr && nrow <= 512) return launch_jacobi_wpp(s, w, nrow, ncol, tol, negl_scale, max_sweeps);
  const bool flow = w.epoch != nullptr;
  const void* fn = flow ? (const void*)jacobi_kernel<NT, TPL, true> : (const void*)jacobi_kernel<NT, TPL, false>;
  static std::atomic<int> cfg_dev{-1}, cfg_blocks{0};  // blocks stored before the device tag
  int dev = 0;
  TT_CUDA_CHECK(cudaGetDevice(&dev));
  if (cfg_dev != dev) {
    int occ_a = 0, occ_b = 0;
    TT_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_a, jacobi_kernel<NT, TPL, true>, NT, 0));
    TT_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_b, jacobi_kernel<NT, TPL, false>, NT, 0));
    cfg_blocks = std::min(occ_a, occ_b) * num_sms();
    cfg_dev = dev;
  }
  int blocks = (int)std::min<int64_t>(ceil_div(npairs, NT / 32), cfg_blocks.load());
  if (blocks < 1) blocks = 1;
  if (flow) TT_CUDA_CHECK(cudaMemsetAsync(w.epoch, 0, (size_t)ncol * sizeof(unsigned), s));
  double* X = w.X;
  int ldx = w.ldx;
  const double* nrm = w.norm;
  unsigned *bar = w.bar, *rot = w.rot, *st = w.status, *ep = w.epoch;
  int* sw = w.sweeps;
  void* args[] = {&X, &nrow, &ncol, &ldx, &tol, &negl_scale, &nrm, &max_sweeps, &bar, &rot, &st, &sw, &ep};
  TT_CUDA_CHECK(cudaLaunchCooperativeKernel(fn, dim3(blocks), dim3(NT), args, 0, s));
  note_launch();
  return TT_OK;
}

int jacobi_svd(cudaStream_t s, SvdWork& w, int nrow, int ncol, double tol, int max_sweeps,
               double delta_scale) {
  // A column with ||x||^2 < delta^2 / (2 ncol) is truncated even after any rotation
  // among such columns (all of them together hold less than delta^2 / 2), so pairs of
  // two such columns are left alone; delta_scale = 0 rotates every pair.
  const double negl_scale = delta_scale > 0.0 ? delta_scale / std::sqrt(2.0 * std::max(ncol, 1)) : 0.0;
  if (ncol <= 0 || nrow <= 0) return TT_OK;
  if (max_sweeps > SvdWork::kMaxSweeps) max_sweeps = SvdWork::kMaxSweeps;
  TT_CUDA_CHECK(cudaMemsetAsync(w.bar, 0, 2 * sizeof(unsigned), s));
  TT_CUDA_CHECK(cudaMemsetAsync(w.rot, 0, SvdWork::kMaxSweeps * sizeof(unsigned), s));
  if (nrow <= 128) return launch_jacobi<64, 4>(s, w, nrow, ncol, tol, negl_scale, max_sweeps);
  if (nrow <= 256) return launch_jacobi<64, 8>(s, w, nrow, ncol, tol, negl_scale, max_sweeps);
  if (nrow <= 512) return launch_jacobi<64, 16>(s, w, nrow, ncol, tol, negl_scale, max_sweeps);
  return launch_jacobi<64, 0>(s, w, nrow, ncol, tol, negl_scale, max_sweeps);
}

int svd_truncate(cudaStream_t s, SvdWork& w, int nrow, int ncol, double delta_scale,
                 int64_t max_rank, double rel_floor) {
  const size_t smem = 2 * (size_t)ncol * sizeof(double);
  if (smem > 200 * 1024) return fail(TT_ERR_UNSUPPORTED, "svd_truncate: bond rank too large");
  static std::atomic<int> configured_dev{-1};
  int dev = 0;
  TT_CUDA_CHECK(cudaGetDevice(&dev));
  if (configured_dev != dev) {
    TT_CUDA_CHECK(cudaFuncSetAttribute(svd_truncate_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    configured_dev = dev;
  }
  svd_truncate_kernel<<<1, 1024, smem, s>>>(w.X, nrow, ncol, w.ldx, w.norm, delta_scale,
                                            (long long)max_rank, rel_floor, w.sigma, w.perm, w.rank,
                                            w.status);
  TT_LAUNCH_CHECK();
  return TT_OK;
}

int certify_full_rank(cudaStream_t s, SvdWork& w, const double* R, int p, int ldr, double delta_scale,
                      double unit, double rel_floor) {
  static std::atomic<int> configured{-1};
  int dev = 0;
  TT_CUDA_CHECK(cudaGetDevice(&dev));
  const size_t smem = 8 * (size_t)p * sizeof(double);
  if (smem > 200 * 1024) return fail(TT_ERR_UNSUPPORTED, "certify_full_rank: rank too large");
  if (configured != dev) {
    TT_CUDA_CHECK(cudaFuncSetAttribute(rinv_colnorm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       200 * 1024));
    configured = dev;
  }
  if (p <= 512) {
    static std::atomic<int> configured_cols{-1};
    if (configured_cols != dev) {
      TT_CUDA_CHECK(cudaFuncSetAttribute(rinv_colnorm_cols_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         200 * 1024));
      TT_CUDA_CHECK(cudaFuncSetAttribute(rinv_colnorm_cols_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         200 * 1024));
      TT_CUDA_CHECK(cudaFuncSetAttribute(rinv_colnorm_cols_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         200 * 1024));
      configured_cols = dev;
    }
    const size_t smem_c = ((size_t)p * 32 + 32) * sizeof(double);
    const unsigned grid = (unsigned)ceil_div(p, kRinvWarps);
    if (p <= 128)
      rinv_colnorm_cols_kernel<4><<<grid, 32 * kRinvWarps, smem_c, s>>>(R, p, ldr, w.sigma);
    else if (p <= 256)
      rinv_colnorm_cols_kernel<8><<<grid, 32 * kRinvWarps, smem_c, s>>>(R, p, ldr, w.sigma);
    else
      rinv_colnorm_cols_kernel<16><<<grid, 32 * kRinvWarps, smem_c, s>>>(R, p, ldr, w.sigma);
  } else {
    rinv_colnorm_kernel<<<(unsigned)ceil_div(p, 8), 256, smem, s>>>(R, p, ldr, w.sigma);
  }
  TT_LAUNCH_CHECK();
  certify_kernel<<<1, 1024, 0, s>>>(R, p, ldr, w.sigma, w.norm, delta_scale, unit, rel_floor, w.rank);
  TT_LAUNCH_CHECK();
  return TT_OK;
}

size_t jacobi_block_smem_gs(int gs, int nrow, int ncol) {
  return (size_t)2 * gs * ((size_t)nrow + ncol) * sizeof(float);
}

size_t jacobi_block_smem(int nrow, int ncol) { return jacobi_block_smem_gs(16, nrow, ncol); }

namespace {

template <int GS, int TPL>
int launch_jacobi_block(cudaStream_t s, SvdWork& w, float* X, int nrow, int ncol, int ldx, float* V,
                        int ldv, int max_sweeps) {
  constexpr int NT = 32 * GS;
  const size_t smem = jacobi_block_smem_gs(GS, nrow, ncol);
  static std::atomic<int> cfg_dev{-1}, cfg_blocks{0};  // blocks stored before the device tag
  int dev = 0;
  TT_CUDA_CHECK(cudaGetDevice(&dev));
  if (cfg_dev != dev) {
    TT_CUDA_CHECK(cudaFuncSetAttribute(jacobi_block_f32_kernel<GS, TPL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       200 * 1024));
    int occ = 0;
    TT_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, jacobi_block_f32_kernel<GS, TPL>, NT,
                                                                200 * 1024));
    cfg_blocks = std::max(1, occ) * num_sms();
    cfg_dev = dev;
  }
  if (V) {
    identity_f32_kernel<<<(unsigned)std::min<int64_t>(ceil_div((int64_t)ncol * ncol, 256), 4096), 256, 0, s>>>(
        V, ncol, ldv);
    TT_LAUNCH_CHECK();
  }
  TT_CUDA_CHECK(cudaMemsetAsync(w.bar, 0, 2 * sizeof(unsigned), s));
  TT_CUDA_CHECK(cudaMemsetAsync(w.rot, 0, SvdWork::kMaxSweeps * sizeof(unsigned), s));
  const int G = (ncol + GS - 1) / GS;
  const int NG = G + (G & 1);
  int blocks = std::min(NG / 2, cfg_blocks.load());
  if (blocks < 1) blocks = 1;
  // 8 sqrt(n) 2^-24: the rounding of an FP32 dot product of n terms is ~sqrt(n) 2^-24
  // of |a| |b|, so a smaller tolerance can keep rotating on noise (it did for n = 2); the
  // kept vectors are re-orthonormalised afterwards, which absorbs this defect
  const float tol = 8.f * std::sqrt((float)std::max(nrow, 1)) * 5.9604645e-8f;
  unsigned *bar = w.bar, *rot = w.rot, *st = w.status;
  int* sw = w.sweeps;
  unsigned* ep = w.epoch;
  if (ep) TT_CUDA_CHECK(cudaMemsetAsync(ep, 0, (size_t)G * sizeof(unsigned), s));
  // pairs of columns below 2^-22 ||x|| / sqrt(2 p) are left alone: that is under the
  // mixed form's resolution floor (2^-22 sigma_1 >= 2^-22 ||x|| / sqrt(p)), FP32
  // rotations cannot make such noise columns orthogonal, and the truncation drops them
  float negl_scale = (float)(1.0 / (1 << 22) / std::sqrt(2.0 * std::max(ncol, 1)));
  const double* nrm = w.norm;
  void* args[] = {&X, &nrow, &ncol, &ldx, &V, &ldv, (void*)&tol, &max_sweeps, &bar, &rot, &st, &sw, &ep,
                  &negl_scale, &nrm};
  TT_CUDA_CHECK(cudaLaunchCooperativeKernel((const void*)jacobi_block_f32_kernel<GS, TPL>, dim3(blocks), dim3(NT),
                                            args, smem, s));
  note_launch();
  return TT_OK;
}

}  // namespace

int jacobi_block_f32(cudaStream_t s, SvdWork& w, float* X, int nrow, int ncol, int ldx, float* V, int ldv,
                     int max_sweeps) {
  if (ncol <= 0 || nrow <= 0) return TT_OK;
  if (max_sweeps > SvdWork::kMaxSweeps) max_sweeps = SvdWork::kMaxSweeps;
  // group size GS: p / (2 GS) CTAs share the work of an outer round
  constexpr int kGroup = 16;
  if (jacobi_block_smem_gs(kGroup, nrow, ncol) > 200 * 1024)
    return fail(TT_ERR_UNSUPPORTED, "jacobi_block_f32: factor too large");
  const int len = std::max(nrow, ncol);  // register chunk: 32 * TPL values per column
  if (len <= 128) return launch_jacobi_block<kGroup, 4>(s, w, X, nrow, ncol, ldx, V, ldv, max_sweeps);
  if (len <= 256) return launch_jacobi_block<kGroup, 8>(s, w, X, nrow, ncol, ldx, V, ldv, max_sweeps);
  return launch_jacobi_block<kGroup, 12>(s, w, X, nrow, ncol, ldx, V, ldv, max_sweeps);
}

template <typename TO>
int svd_left_vectors(cudaStream_t s, const SvdWork& w, int nrow, int r, TO* U) {
  const int64_t total = (int64_t)nrow * r;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(total, 256), 4096));
  svd_left_kernel<TO><<<blocks, 256, 0, s>>>(w.X, nrow, w.ldx, w.perm, w.sigma, r, U);
  TT_LAUNCH_CHECK();
  return TT_OK;
}

// ---------------------------------------------------------------- batched launchers
int certify_batched(cudaStream_t s, int nj, const SvdJob* d_jobs, int n_max, double unit, double rel_floor) {
  if (nj <= 0 || n_max <= 0) return TT_OK;
  const size_t smem = 8 * (size_t)n_max * sizeof(double);
  if (smem > 200 * 1024) return fail(TT_ERR_UNSUPPORTED, "certify_batched: rank too large");
  static std::atomic<int> configured{-1};
  int dev = 0;
  TT_CUDA_CHECK(cudaGetDevice(&dev));
  if (configured != dev) {
    TT_CUDA_CHECK(cudaFuncSetAttribute(rinv_colnorm_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       200 * 1024));
    configured = dev;
  }
  if (n_max <= 640) {
    static std::atomic<int> configured_cols{-1};
    if (configured_cols != dev) {
      TT_CUDA_CHECK(cudaFuncSetAttribute(rinv_colnorm_cols_batched_kernel<4>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
      TT_CUDA_CHECK(cudaFuncSetAttribute(rinv_colnorm_cols_batched_kernel<8>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
      TT_CUDA_CHECK(cudaFuncSetAttribute(rinv_colnorm_cols_batched_kernel<16>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
      TT_CUDA_CHECK(cudaFuncSetAttribute(rinv_colnorm_cols_batched_kernel<20>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
      configured_cols = dev;
    }
    const size_t smem_c = ((size_t)n_max * 32 + 32) * sizeof(double);
    const dim3 grid((unsigned)ceil_div(n_max, kRinvWarps), (unsigned)nj);
    if (n_max <= 128)
      rinv_colnorm_cols_batched_kernel<4><<<grid, 32 * kRinvWarps, smem_c, s>>>(d_jobs);
    else if (n_max <= 256)
      rinv_colnorm_cols_batched_kernel<8><<<grid, 32 * kRinvWarps, smem_c, s>>>(d_jobs);
    else if (n_max <= 512)
      rinv_colnorm_cols_batched_kernel<16><<<grid, 32 * kRinvWarps, smem_c, s>>>(d_jobs);
    else
      rinv_colnorm_cols_batched_kernel<20><<<grid, 32 * kRinvWarps, smem_c, s>>>(d_jobs);
  } else {
    rinv_colnorm_batched_kernel<<<dim3((unsigned)ceil_div(n_max, 8), (unsigned)nj), 256, smem, s>>>(d_jobs);
  }
  TT_LAUNCH_CHECK();
  certify_batched_kernel<<<nj, 1024, 0, s>>>(d_jobs, unit, rel_floor);
  TT_LAUNCH_CHECK();
  return TT_OK;
}

namespace {

template <typename K, typename... Args>
int launch_cluster(cudaStream_t s, K kernel, int cs, int nj, int nt, size_t smem, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(nj * cs));
  cfg.blockDim = dim3((unsigned)nt);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  TT_CUDA_CHECK(cudaLaunchKernelEx(&cfg, kernel, args...));
  note_launch();
  return TT_OK;
}

template <typename K>
int allow_cluster16(K kernel) {
  TT_CUDA_CHECK(cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  return TT_OK;
}

template <int CS>
int f64_cluster(cudaStream_t s, int nj, const SvdJob* d_jobs, int n_max, int skip, int max_sweeps) {
  if (CS > 8) {
    static std::atomic<int> configured{-1};
    int dev = 0;
    TT_CUDA_CHECK(cudaGetDevice(&dev));
    if (configured != dev) {
      TT_TRY(allow_cluster16(jacobi_f64_cluster_kernel<256, 4, CS>));
      TT_TRY(allow_cluster16(jacobi_f64_cluster_kernel<256, 8, CS>));
      TT_TRY(allow_cluster16(jacobi_f64_cluster_kernel<256, 16, CS>));
      TT_TRY(allow_cluster16(jacobi_f64_cluster_kernel<256, 0, CS>));
      configured = dev;
    }
  }
  if (n_max <= 128)
    return launch_cluster(s, jacobi_f64_cluster_kernel<256, 4, CS>, CS, nj, 256, 0, d_jobs, skip, max_sweeps);
  if (n_max <= 256)
    return launch_cluster(s, jacobi_f64_cluster_kernel<256, 8, CS>, CS, nj, 256, 0, d_jobs, skip, max_sweeps);
  if (n_max <= 512)
    return launch_cluster(s, jacobi_f64_cluster_kernel<256, 16, CS>, CS, nj, 256, 0, d_jobs, skip,
                          max_sweeps);
  return launch_cluster(s, jacobi_f64_cluster_kernel<256, 0, CS>, CS, nj, 256, 0, d_jobs, skip, max_sweeps);
}

template <int CS>
int f32_cluster(cudaStream_t s, int nj, const SvdJob* d_jobs, int n_max, int max_sweeps) {
  if (CS > 8) {
    static std::atomic<int> configured{-1};
    int dev = 0;
    TT_CUDA_CHECK(cudaGetDevice(&dev));
    if (configured != dev) {
      TT_TRY(allow_cluster16(jacobi_f32rr_cluster_kernel<256, 4, CS>));
      TT_TRY(allow_cluster16(jacobi_f32rr_cluster_kernel<256, 8, CS>));
      TT_TRY(allow_cluster16(jacobi_f32rr_cluster_kernel<256, 16, CS>));
      TT_TRY(allow_cluster16(jacobi_f32rr_cluster_kernel<256, 20, CS>));
      configured = dev;
    }
  }
  if (n_max <= 128)
    return launch_cluster(s, jacobi_f32rr_cluster_kernel<256, 4, CS>, CS, nj, 256, 0, d_jobs, max_sweeps);
  if (n_max <= 256)
    return launch_cluster(s, jacobi_f32rr_cluster_kernel<256, 8, CS>, CS, nj, 256, 0, d_jobs, max_sweeps);
  if (n_max <= 512)
    return launch_cluster(s, jacobi_f32rr_cluster_kernel<256, 16, CS>, CS, nj, 256, 0, d_jobs, max_sweeps);
  return launch_cluster(s, jacobi_f32rr_cluster_kernel<256, 20, CS>, CS, nj, 256, 0, d_jobs, max_sweeps);
}

}  // namespace

int svd_cluster_size(int n, bool fp64) {
  // about two to four pairs per warp and round, 8 warps per CTA; the FP64 kernel is bound
  // by the FP64 pipe of its SMs and gains from 16 CTAs on the largest factors, the FP32
  // one (latency-bound, many jobs side by side) does not
  if (n <= 64) return 1;
  if (n <= 128) return 2;
  if (n <= 256) return 4;
  if (n <= 320 || !fp64) return 8;
  return 16;
}

int jacobi_f64_batched(cudaStream_t s, int nj, const SvdJob* d_jobs, int n_max, bool skip,
                       int max_sweeps, int cs) {
  if (nj <= 0 || n_max <= 0) return TT_OK;
  switch (cs) {
    case 1: return f64_cluster<1>(s, nj, d_jobs, n_max, skip ? 1 : 0, max_sweeps);
    case 2: return f64_cluster<2>(s, nj, d_jobs, n_max, skip ? 1 : 0, max_sweeps);
    case 4: return f64_cluster<4>(s, nj, d_jobs, n_max, skip ? 1 : 0, max_sweeps);
    case 8: return f64_cluster<8>(s, nj, d_jobs, n_max, skip ? 1 : 0, max_sweeps);
    case 16: return f64_cluster<16>(s, nj, d_jobs, n_max, skip ? 1 : 0, max_sweeps);
  }
  return fail(TT_ERR_ARG, "jacobi_f64_batched: cluster size");
}

int jacobi_f32_batched(cudaStream_t s, int nj, const SvdJob* d_jobs, int n_max, int max_sweeps, int cs) {
  if (nj <= 0 || n_max <= 0) return TT_OK;
  switch (cs) {
    case 1: return f32_cluster<1>(s, nj, d_jobs, n_max, max_sweeps);
    case 2: return f32_cluster<2>(s, nj, d_jobs, n_max, max_sweeps);
    case 4: return f32_cluster<4>(s, nj, d_jobs, n_max, max_sweeps);
    case 8: return f32_cluster<8>(s, nj, d_jobs, n_max, max_sweeps);
    case 16: return f32_cluster<16>(s, nj, d_jobs, n_max, max_sweeps);
  }
  return fail(TT_ERR_ARG, "jacobi_f32_batched: cluster size");
}

int svd_truncate_batched(cudaStream_t s, int nj, const SvdJob* d_jobs, int n_max, int64_t max_rank,
                         double rel_floor) {
  if (nj <= 0 || n_max <= 0) return TT_OK;
  const size_t smem = 2 * (size_t)n_max * sizeof(double);
  if (smem > 200 * 1024) return fail(TT_ERR_UNSUPPORTED, "svd_truncate_batched: bond rank too large");
  static std::atomic<int> configured{-1};
  int dev = 0;
  TT_CUDA_CHECK(cudaGetDevice(&dev));
  if (configured != dev) {
    TT_CUDA_CHECK(cudaFuncSetAttribute(svd_truncate_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       200 * 1024));
    configured = dev;
  }
  svd_truncate_batched_kernel<<<nj, 1024, smem, s>>>(d_jobs, (long long)max_rank, rel_floor);
  TT_LAUNCH_CHECK();
  return TT_OK;
}

template <typename TO>
int svd_left_batched(cudaStream_t s, int nj, const SvdJob* d_jobs, int64_t max_elems) {
  if (nj <= 0 || max_elems <= 0) return TT_OK;
  svd_left_batched_kernel<TO>
      <<<dim3((unsigned)std::min<int64_t>(ceil_div(max_elems, 256), 1024), (unsigned)nj), 256, 0, s>>>(d_jobs);
  TT_LAUNCH_CHECK();
  return TT_OK;
}

template int svd_left_batched<double>(cudaStream_t, int, const SvdJob*, int64_t);
template int svd_left_batched<float>(cudaStream_t, int, const SvdJob*, int64_t);
template int svd_left_vectors<double>(cudaStream_t, const SvdWork&, int, int, double*);
template int svd_left_vectors<float>(cudaStream_t, const SvdWork&, int, int, float*);

}  // namespace tt
