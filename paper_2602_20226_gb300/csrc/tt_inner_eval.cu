// TT inner product by the environment sweep, its adjoint, and batched evaluation.
//
// <x, y>: E_0 = 1, E_k = sum_i X_k(i)^T E_{k-1} Y_k(i) (r^x_k x r^y_k), accumulated in
// FP64 for both dtypes.  Each site is two GEMMs: T = E_{k-1} Y_k (Y_k as
// r^y_{k-1} x (d r^y_k)) and E_k = X_k'^T T' with X_k' = (r^x_{k-1} d) x r^x_k.
//
// Evaluation: each thread owns one sample and keeps its row vector
// v = G_1[:, i_1, :] ... G_k[:, i_k, :] in shared memory (column-per-thread, so
// accesses are conflict-free); the cores are read through the read-only cache
// where a warp's lanes share at most d distinct rows per load.
#include <type_traits>
#include <vector>

#include "tt_gemm.cuh"
#include "tt_inner_eval.cuh"

namespace tt {

namespace {

__global__ void set_scalar_kernel(double* p, double v) { *p = v; }

// values[s] for samples [blockIdx.x * S, ...).  vbuf: two (rmax x S) planes of T.
template <typename T, int JB>
__global__ void eval_kernel(EvalParams<T> P, const uint8_t* __restrict__ digits, long long n,
                            T* __restrict__ values, unsigned* status) {
  extern __shared__ unsigned char smem_raw[];
  T* buf = reinterpret_cast<T*>(smem_raw);
  const int S = blockDim.x;
  const int tid = threadIdx.x;
  const long long smp = (long long)blockIdx.x * S + tid;
  const bool active = smp < n;
  T* cur = buf;
  T* nxt = buf + (size_t)P.rmax * S;
  cur[tid] = T(1);
  for (int k = 0; k < P.L; ++k) {
    const int r0 = P.r[k], r1 = P.r[k + 1], d = P.d[k];
    const T* G = P.g[k];
    int dig = active ? (int)digits[smp * P.L + k] : 0;
    if (dig >= d) {
      if (status) atomicOr(status, (unsigned)ST_BAD_INDEX);
      dig = 0;
    }
    for (int j0 = 0; j0 < r1; j0 += JB) {
      T acc[JB];
#pragma unroll
      for (int t = 0; t < JB; ++t) acc[t] = T(0);
      const int jn = min(JB, r1 - j0);
      for (int a = 0; a < r0; ++a) {
        const T v = cur[(size_t)a * S + tid];
        const T* grow = G + ((long long)a * d + dig) * r1 + j0;
#pragma unroll
        for (int t = 0; t < JB; ++t)
          if (t < jn) acc[t] = fma(v, __ldg(grow + t), acc[t]);
      }
#pragma unroll
      for (int t = 0; t < JB; ++t)
        if (t < jn) nxt[(size_t)(j0 + t) * S + tid] = acc[t];
    }
    T* tmp = cur;
    cur = nxt;
    nxt = tmp;
  }
  if (active) values[smp] = cur[tid];
}

// Staged form (used when a core fits in shared memory next to the row buffers): per site the
// CTA copies G_k once into shared memory (rows (a, i) padded to a multiple of 16 bytes plus
// 16 bytes, so the d digit slices of a row start in different banks), and every thread forms
// its sample's next row vector from vector loads of the staged core: one 16-byte shared load
// feeds 4 (FP32) or 2 (FP64) FMAs, where the direct form issued one global load per FMA.
// The CTA's digits are staged once (S x L contiguous bytes).
template <typename T>
__host__ __device__ constexpr int eval_row_pad(int r1) {
  return sizeof(T) == 4 ? ((r1 + 3) & ~3) + 4 : ((r1 + 1) & ~1) + 2;
}

// Copies the CTA's nb digit bytes into shared memory: 16-byte loads when the source is
// 16-byte aligned, all of a thread's loads issued before its stores.
__device__ __forceinline__ void stage_digits(const uint8_t* __restrict__ src, long long nb, uint8_t* __restrict__ dst) {
  const int S = blockDim.x;
  long long done = 0;
  if ((reinterpret_cast<uintptr_t>(src) & 15) == 0 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
    const long long n16 = nb / 16;
    const uint4* s4 = reinterpret_cast<const uint4*>(src);
    uint4* d4 = reinterpret_cast<uint4*>(dst);
    for (long long base = threadIdx.x; base < n16; base += (long long)S * 4) {
      uint4 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const long long q = base + (long long)u * S;
        if (q < n16) v[u] = __ldg(s4 + q);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const long long q = base + (long long)u * S;
        if (q < n16) d4[q] = v[u];
      }
    }
    done = n16 * 16;
  }
  for (long long e = done + threadIdx.x; e < nb; e += S) dst[e] = src[e];
}

// Copies core G (rows = r0 d rows of r1 values, row-major) into shared memory: row-major with
// row stride ldst, or transposed (row (c d + i) holds G[:, i, c], stride ldst).  Each thread
// issues U loads before its first store, so staging a core costs a few L2 latencies rather
// than one per element a thread copies.
template <typename T, int U>
__device__ __forceinline__ void stage_core(const T* __restrict__ G, int r0, int d, int r1, T* __restrict__ stage,
                                           int ldst, bool transpose) {
  const int total = r0 * d * r1;
  const int S = blockDim.x;
  for (int base = threadIdx.x; base < total; base += S * U) {
    T v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = base + u * S;
      v[u] = e < total ? __ldg(G + e) : T(0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = base + u * S;
      if (e < total) {
        const int row = e / r1, c = e - row * r1;
        if (!transpose) {
          stage[row * ldst + c] = v[u];
        } else {
          const int a = row / d, i = row - a * d;
          stage[(c * d + i) * ldst + a] = v[u];
        }
      }
    }
  }
}

// ONE: every output block fits one pass (JB >= every r_k): a thread reads only its own column
// of the row buffer and writes it after its last read, so the row vector is updated in place
// (one buffer: a third more CTAs per SM at rank 64).
template <typename T, int JB, bool ONE>
__global__ void eval_staged_kernel(EvalParams<T> P, const uint8_t* __restrict__ digits, long long n,
                                   T* __restrict__ values, unsigned* status, int stage_elems) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int S = blockDim.x;
  const int tid = threadIdx.x;
  T* cur = reinterpret_cast<T*>(smem_raw);
  T* nxt = ONE ? cur : cur + (size_t)P.rmax * S;
  T* stage = (ONE ? cur : nxt) + (size_t)P.rmax * S;
  uint8_t* dg = reinterpret_cast<uint8_t*>(stage + stage_elems + JB);
  const long long s0 = (long long)blockIdx.x * S;
  const long long smp = s0 + tid;
  const bool active = smp < n;
  {
    const long long nb = (long long)min((long long)S, n - s0) * P.L;
    const uint8_t* src = digits + s0 * P.L;
    stage_digits(src, nb, dg);
  }
  cur[tid] = T(1);
  constexpr int VW = 16 / sizeof(T);  // elements per 16-byte load
  using V = std::conditional_t<sizeof(T) == 4, float4, double2>;
  for (int k = 0; k < P.L; ++k) {
    const int r0 = P.r[k], r1 = P.r[k + 1], d = P.d[k];
    const int r1p = eval_row_pad<T>(r1);
    __syncthreads();  // the previous site is done with the stage; digits are staged
    stage_core<T, 16 / (sizeof(T) / 4)>(P.g[k], r0, d, r1, stage, r1p, false);
    __syncthreads();
    int dig = active ? (int)dg[tid * P.L + k] : 0;
    if (dig >= d) {
      if (status) atomicOr(status, (unsigned)ST_BAD_INDEX);
      dig = 0;
    }
    for (int j0 = 0; j0 < r1; j0 += JB) {
      T acc[JB];
#pragma unroll
      for (int t = 0; t < JB; ++t) acc[t] = T(0);
      for (int a = 0; a < r0; ++a) {
        const T v = cur[(size_t)a * S + tid];
        const V* g = reinterpret_cast<const V*>(stage + (size_t)(a * d + dig) * r1p + j0);
#pragma unroll
        for (int q = 0; q < JB / VW; ++q) {
          const V w = g[q];
          if constexpr (VW == 4) {
            acc[4 * q + 0] = fma(v, w.x, acc[4 * q + 0]);
            acc[4 * q + 1] = fma(v, w.y, acc[4 * q + 1]);
            acc[4 * q + 2] = fma(v, w.z, acc[4 * q + 2]);
            acc[4 * q + 3] = fma(v, w.w, acc[4 * q + 3]);
          } else {
            acc[2 * q + 0] = fma(v, w.x, acc[2 * q + 0]);
            acc[2 * q + 1] = fma(v, w.y, acc[2 * q + 1]);
          }
        }
      }
      const int jn = min(JB, r1 - j0);
#pragma unroll
      for (int t = 0; t < JB; ++t)
        if (t < jn) nxt[(size_t)(j0 + t) * S + tid] = acc[t];
    }
    if constexpr (!ONE) {
      T* tmp = cur;
      cur = nxt;
      nxt = tmp;
    }
  }
  if (active) values[smp] = cur[tid];
}

// ------------------------------------------------------------------ eval backward
// The adjoint of evaluation is, per site k and digit i, a contraction over samples:
//   dG_k[:, i, :] = sum_{s : i_k^s = i} w_s p_{k,s}^T q_{k,s}
// with p_{k,s} = G_1[:, i_1^s, :] ... G_{k-1}[:, i_{k-1}^s, :] (the row vector in front of
// site k) and q_{k,s} = G_{k+1}[:, i_{k+1}^s, :] ... G_L[:, i_L^s, :] (the column vector after
// it).  For a chunk of C samples, eval_states_kernel stores every p_k and q_k (state-major,
// [j][C], so that a thread per sample writes coalesced rows), one CTA of samples sweeping
// left to right and one right to left in the same launch; eval_bwd_accum_kernel then forms
// the per-site sums as (r_{k-1} x samples) . (samples x r_k) products, the samples of each
// digit taken from a per-tile list, and adds them into FP64 accumulators.

// Offsets (elements) of the prefix and suffix states of site k inside a chunk's store.
__device__ __forceinline__ long long prefix_off(const int* r, int k, long long C) {
  long long o = 0;
  for (int j = 0; j < k; ++j) o += r[j];
  return o * C;
}
__device__ __forceinline__ long long suffix_off(const int* r, int L, int k, long long C) {
  long long o = 0;
  for (int j = 0; j < L; ++j) o += r[j];  // the prefix block comes first
  for (int j = 0; j < k; ++j) o += r[j + 1];
  return o * C;
}

// blockIdx.y = 0: prefixes (left to right), 1: suffixes (right to left).  Same staging and
// inner loop as eval_staged_kernel; for the suffixes the core is staged transposed
// (row (b, i) holds G[:, i, b]), so that both directions form out = cur . stage-rows.
template <typename T, int JB, bool ONE>
__global__ void eval_states_kernel(EvalParams<T> P, const uint8_t* __restrict__ digits, long long n,
                                   T* __restrict__ states, long long C, int stage_elems) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int S = blockDim.x;
  const int tid = threadIdx.x;
  const bool suffix = blockIdx.y == 1;
  T* cur = reinterpret_cast<T*>(smem_raw);
  T* nxt = ONE ? cur : cur + (size_t)P.rmax * S;  // ONE: in place, as in eval_staged_kernel
  T* stage = (ONE ? cur : nxt) + (size_t)P.rmax * S;
  uint8_t* dg = reinterpret_cast<uint8_t*>(stage + stage_elems + JB);
  const long long s0 = (long long)blockIdx.x * S;
  const long long smp = s0 + tid;
  const bool active = smp < n;
  {
    const long long nb = (long long)min((long long)S, n - s0) * P.L;
    const uint8_t* src = digits + s0 * P.L;
    stage_digits(src, nb, dg);
  }
  cur[tid] = T(1);
  constexpr int VW = 16 / sizeof(T);
  using V = std::conditional_t<sizeof(T) == 4, float4, double2>;
  const int L = P.L;
  for (int step = 0; step < L; ++step) {
    const int k = suffix ? L - 1 - step : step;
    const int r0 = P.r[k], r1 = P.r[k + 1], d = P.d[k];
    const int rin = suffix ? r1 : r0, rout = suffix ? r0 : r1;
    // the state in front of site k (prefix) or after it (suffix)
    if (active) {
      T* dst = states + (suffix ? suffix_off(P.r, L, k, C) : prefix_off(P.r, k, C)) + smp;
      for (int j = 0; j < rin; ++j) dst[(long long)j * C] = cur[(size_t)j * S + tid];
    }
    if (step == L - 1) break;  // the full product is not needed
    const int routp = eval_row_pad<T>(rout);
    __syncthreads();
    stage_core<T, 16 / (sizeof(T) / 4)>(P.g[k], r0, d, r1, stage, routp, suffix);
    __syncthreads();
    int dig = active ? (int)dg[tid * L + k] : 0;
    if (dig >= d) dig = 0;  // the accumulation skips such samples at this site
    for (int j0 = 0; j0 < rout; j0 += JB) {
      T acc[JB];
#pragma unroll
      for (int t = 0; t < JB; ++t) acc[t] = T(0);
      for (int a = 0; a < rin; ++a) {
        const T v = cur[(size_t)a * S + tid];
        const V* g = reinterpret_cast<const V*>(stage + (size_t)(a * d + dig) * routp + j0);
#pragma unroll
        for (int q = 0; q < JB / VW; ++q) {
          const V w = g[q];
          if constexpr (VW == 4) {
            acc[4 * q + 0] = fma(v, w.x, acc[4 * q + 0]);
            acc[4 * q + 1] = fma(v, w.y, acc[4 * q + 1]);
            acc[4 * q + 2] = fma(v, w.z, acc[4 * q + 2]);
            acc[4 * q + 3] = fma(v, w.w, acc[4 * q + 3]);
          } else {
            acc[2 * q + 0] = fma(v, w.x, acc[2 * q + 0]);
            acc[2 * q + 1] = fma(v, w.y, acc[2 * q + 1]);
          }
        }
      }
      const int jn = min(JB, rout - j0);
#pragma unroll
      for (int t = 0; t < JB; ++t)
        if (t < jn) nxt[(size_t)(j0 + t) * S + tid] = acc[t];
    }
    if constexpr (!ONE) {
      T* tmp = cur;
      cur = nxt;
      nxt = tmp;
    }
  }
}

// Per-site accumulation over one slice of a chunk's samples.  Grid: x = sample slice,
// y = (a, b) tile of 64 x 64, z = site * digit groups + group.  128 threads, each owning an
// 8 x 4 block of the tile for DG digits (registers); samples go through shared memory in
// tiles of 32 (prefix scaled by w_s, both transposed to sample-major rows), and for each
// digit of the group the CTA walks only the samples that carry it (a list built by ballot),
// so the work is r_{k-1} r_k multiply-adds per sample and site.  The slice's sums (in T)
// are added into the FP64 accumulator acc[k] with one atomic per entry.
constexpr int kAccTile = 64, kAccK = 32;

struct SiteMask {
  unsigned char on[TT_MAX_SITES];
};

template <typename T, int DG>
__global__ void __launch_bounds__(128) eval_bwd_accum_kernel(EvalParams<T> P, SiteMask want,
                                                            const uint8_t* __restrict__ digits, const T* __restrict__ w,
                                                            long long n, const T* __restrict__ states, long long C,
                                                            long long slice, double* __restrict__ acc) {
  constexpr int PS = kAccTile + 4;  // row stride of the staged tiles (16-byte rows, fewer conflicts)
  __shared__ __align__(16) T Ps[kAccK][PS];
  __shared__ __align__(16) T Qs[kAccK][PS];
  __shared__ int list[DG][kAccK];
  __shared__ int cnt[DG];
  const int L = P.L;
  const int tid = threadIdx.x;
  int kz = blockIdx.z;
  int k = 0;
  // site and digit group of this CTA
  {
    int z = kz;
    for (k = 0; k < L; ++k) {
      const int g = (P.d[k] + DG - 1) / DG;
      if (z < g) break;
      z -= g;
    }
    kz = z;  // digit group within site k
  }
  if (k >= L || !want.on[k]) return;
  const int r0 = P.r[k], r1 = P.r[k + 1], d = P.d[k];
  const int ntb = (r1 + kAccTile - 1) / kAccTile;
  const int a0 = (blockIdx.y / ntb) * kAccTile, b0 = (blockIdx.y % ntb) * kAccTile;
  if (a0 >= r0) return;
  const int i0 = kz * DG;
  const T* Pk = states + prefix_off(P.r, k, C);
  const T* Qk = states + suffix_off(P.r, L, k, C);
  const long long sb = (long long)blockIdx.x * slice, se = min(n, sb + slice);
  const int ta = tid >> 4, tb = tid & 15;  // 8 x 16 threads: rows ta*8.., columns tb*4..
  T accr[DG][8][4];
#pragma unroll
  for (int g = 0; g < DG; ++g)
#pragma unroll
    for (int x = 0; x < 8; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) accr[g][x][y] = T(0);
  for (long long t0 = sb; t0 < se; t0 += kAccK) {
    const int kt = (int)min((long long)kAccK, se - t0);
    __syncthreads();  // the previous tile is consumed
    // stage p (times w) and q: element e -> (row j, sample s), coalesced along samples; a
    // thread issues the loads of four elements before storing any
    constexpr int SU = 4;
    for (int e0 = tid; e0 < kAccTile * kAccK; e0 += 128 * SU) {
      T pv[SU], qv[SU], wv[SU];
#pragma unroll
      for (int u = 0; u < SU; ++u) {
        const int e = e0 + 128 * u, j = e / kAccK, s = e - j * kAccK;
        pv[u] = qv[u] = wv[u] = T(0);
        if (s < kt) {
          if (a0 + j < r0) pv[u] = __ldg(Pk + (long long)(a0 + j) * C + t0 + s);
          if (b0 + j < r1) qv[u] = __ldg(Qk + (long long)(b0 + j) * C + t0 + s);
          wv[u] = __ldg(w + t0 + s);
        }
      }
#pragma unroll
      for (int u = 0; u < SU; ++u) {
        const int e = e0 + 128 * u, j = e / kAccK, s = e - j * kAccK;
        Ps[s][j] = pv[u] * wv[u];
        Qs[s][j] = qv[u];
      }
    }
    if (tid < 32) {
      const int dgt = tid < kt ? (int)digits[(t0 + tid) * L + k] : -1;
#pragma unroll
      for (int g = 0; g < DG; ++g) {
        const unsigned m = __ballot_sync(0xffffffffu, dgt == i0 + g && i0 + g < d);
        if (dgt == i0 + g && i0 + g < d) list[g][__popc(m & ((1u << tid) - 1u))] = tid;
        if (tid == 0) cnt[g] = __popc(m);
      }
    }
    __syncthreads();
#pragma unroll
    for (int g = 0; g < DG; ++g) {
      const int c = cnt[g];
      for (int q = 0; q < c; ++q) {
        const int s = list[g][q];
        T pa[8], qb[4];
        if constexpr (sizeof(T) == 4) {
          const float4 u0 = *reinterpret_cast<const float4*>(&Ps[s][ta * 8]);
          const float4 u1 = *reinterpret_cast<const float4*>(&Ps[s][ta * 8 + 4]);
          const float4 v0 = *reinterpret_cast<const float4*>(&Qs[s][tb * 4]);
          pa[0] = u0.x; pa[1] = u0.y; pa[2] = u0.z; pa[3] = u0.w;
          pa[4] = u1.x; pa[5] = u1.y; pa[6] = u1.z; pa[7] = u1.w;
          qb[0] = v0.x; qb[1] = v0.y; qb[2] = v0.z; qb[3] = v0.w;
        } else {
#pragma unroll
          for (int x = 0; x < 8; x += 2) {
            const double2 u = *reinterpret_cast<const double2*>(&Ps[s][ta * 8 + x]);
            pa[x] = u.x;
            pa[x + 1] = u.y;
          }
#pragma unroll
          for (int y = 0; y < 4; y += 2) {
            const double2 v = *reinterpret_cast<const double2*>(&Qs[s][tb * 4 + y]);
            qb[y] = v.x;
            qb[y + 1] = v.y;
          }
        }
#pragma unroll
        for (int x = 0; x < 8; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) accr[g][x][y] = fma(pa[x], qb[y], accr[g][x][y]);
      }
    }
  }
  double* acck = acc;
  for (int j = 0; j < k; ++j) acck += (size_t)P.r[j] * P.d[j] * P.r[j + 1];
#pragma unroll
  for (int g = 0; g < DG; ++g) {
    const int i = i0 + g;
    if (i >= d) continue;
#pragma unroll
    for (int x = 0; x < 8; ++x) {
      const int a = a0 + ta * 8 + x;
      if (a >= r0) continue;
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        const int b = b0 + tb * 4 + y;
        if (b < r1 && accr[g][x][y] != T(0)) atomicAdd(acck + ((size_t)a * d + i) * r1 + b, (double)accr[g][x][y]);
      }
    }
  }
}

// Backward of evaluation for one site k: dG_k[a, i, b] += sum_s w_s P_s[a] Sf_s[b] [i_k^s == i].
// prefixes P (n x r0) and suffixes Sf (n x r1) are given row-major in FP64.
template <typename T>
__global__ void eval_bwd_site_kernel(const double* __restrict__ Pm, const double* __restrict__ Sm,
                                     const T* __restrict__ w, const uint8_t* __restrict__ digits,
                                     int L, int k, long long n, int r0, int d, int r1,
                                     double* __restrict__ acc /* r0 x d x r1 */) {
  // each CTA covers a chunk of samples and a tile of (a, b); accumulate then atomicAdd
  const int a = blockIdx.y;
  const long long chunk = (n + gridDim.x - 1) / gridDim.x;
  const long long s0 = blockIdx.x * chunk, s1 = min(n, s0 + chunk);
  for (int b = threadIdx.x; b < r1; b += blockDim.x) {
    double loc[TT_MAX_MODE];
    for (int i = 0; i < d; ++i) loc[i] = 0.0;
    for (long long s = s0; s < s1; ++s) {
      const int i = digits[s * L + k];
      if (i < d) loc[i] += (double)w[s] * Pm[s * r0 + a] * Sm[s * r1 + b];
    }
    for (int i = 0; i < d; ++i)
      if (loc[i] != 0.0) atomicAdd(acc + ((size_t)a * d + i) * r1 + b, loc[i]);
  }
}

// prefix/suffix step:  out[s, :] = in[s, :] * G[:, i_s, :]   (prefix, left to right)
//                      out[s, :] = G[:, i_s, :] * in[s, :]^T (suffix, right to left)
template <typename T>
__global__ void eval_step_kernel(const T* __restrict__ G, int r0, int d, int r1,
                                 const uint8_t* __restrict__ digits, int L, int k, long long n,
                                 const double* __restrict__ in, double* __restrict__ out,
                                 bool suffix) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int rout = suffix ? r0 : r1;
  if (e >= n * rout) return;
  const long long s = e / rout;
  const int j = (int)(e % rout);
  int i = digits[s * L + k];
  if (i >= d) i = 0;
  double acc = 0.0;
  if (!suffix) {
    for (int a = 0; a < r0; ++a) acc += in[s * r0 + a] * (double)G[((long long)a * d + i) * r1 + j];
  } else {
    for (int b = 0; b < r1; ++b) acc += (double)G[((long long)j * d + i) * r1 + b] * in[s * r1 + b];
  }
  out[e] = acc;
}

__global__ void fill_ones_kernel(double* p, long long n) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e < n) p[e] = 1.0;
}

template <typename T>
__global__ void add_into_kernel(const double* src, long long n, T* dst) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e < n) dst[e] += (T)src[e];
}

}  // namespace

// ------------------------------------------------------------------ inner
// The adjoint keeps the left environments only at every c-th site (c = ceil(sqrt(L))) and
// recomputes those of one segment at a time during the right-to-left sweep: O(sqrt(L))
// environments in memory instead of L, for one extra left sweep of GEMMs.
inline int env_segment(int L) {
  int c = 1;
  while (c * c < L) ++c;
  return c;
}

size_t inner_workspace_bytes(const tt_train* x, const tt_train* y) {
  int64_t env = 1, tb = 1;
  for (int k = 0; k <= x->L; ++k) env = std::max<int64_t>(env, x->ranks[k] * y->ranks[k]);
  for (int k = 0; k < x->L; ++k) {
    tb = std::max<int64_t>(tb, x->ranks[k] * (int64_t)x->d[k] * y->ranks[k + 1]);
    tb = std::max<int64_t>(tb, y->ranks[k] * (int64_t)x->d[k] * x->ranks[k + 1]);
  }
  const int c = env_segment(x->L);
  const int64_t ncp = (x->L + c - 1) / c;
  // forward: 2 env + 1 T; backward: checkpoints + one segment of left envs + 2 right envs + 3 T
  return (size_t)((ncp + c + 2) * env + 3 * tb + 64) * sizeof(double) + 1024;
}

template <typename TX, typename TY>
int inner_impl(const tt_train* x, const tt_train* y, double* out, void* ws, size_t ws_bytes,
               cudaStream_t s) {
  if (ws_bytes < inner_workspace_bytes(x, y)) return fail(TT_ERR_WORKSPACE, "tt_inner: workspace too small");
  const int L = x->L;
  int64_t env = 1, tb = 1;
  for (int k = 0; k <= L; ++k) env = std::max<int64_t>(env, x->ranks[k] * y->ranks[k]);
  for (int k = 0; k < L; ++k) tb = std::max<int64_t>(tb, x->ranks[k] * (int64_t)x->d[k] * y->ranks[k + 1]);
  double* E = static_cast<double*>(ws);
  double* E2 = E + env;
  double* Tb = E2 + env;
  set_scalar_kernel<<<1, 1, 0, s>>>(E, 1.0);
  TT_LAUNCH_CHECK();
  for (int k = 0; k < L; ++k) {
    const int rx0 = (int)x->ranks[k], rx1 = (int)x->ranks[k + 1];
    const int ry0 = (int)y->ranks[k], ry1 = (int)y->ranks[k + 1], d = x->d[k];
    const TX* X = static_cast<const TX*>(x->cores[k]);
    const TY* Y = static_cast<const TY*>(y->cores[k]);
    // T (rx0 x d ry1) = E (rx0 x ry0) Y (ry0 x d ry1)
    TT_TRY((gemm<double, TY, double>(s, rx0, d * ry1, ry0, 1.0, E, ry0, 1, Y, (int64_t)d * ry1, 1,
                                     0.0, Tb, (int64_t)d * ry1, 1)));
    // E2 (rx1 x ry1) = X'^T ((rx1) x (rx0 d)) T' ((rx0 d) x ry1)
    TT_TRY((gemm<TX, double, double>(s, rx1, ry1, rx0 * d, 1.0, X, 1, rx1, Tb, ry1, 1, 0.0, E2, ry1, 1)));
    std::swap(E, E2);
  }
  TT_CUDA_CHECK(cudaMemcpyAsync(out, E, sizeof(double), cudaMemcpyDeviceToHost, s));
  TT_CUDA_CHECK(cudaStreamSynchronize(s));
  return TT_OK;
}

template <typename TX, typename TY>
int inner_backward_impl(const tt_train* x, const tt_train* y, double dout, tt_train* dx,
                        tt_train* dy, void* ws, size_t ws_bytes, cudaStream_t s) {
  if (ws_bytes < inner_workspace_bytes(x, y)) return fail(TT_ERR_WORKSPACE, "tt_inner_backward: workspace too small");
  const int L = x->L;
  int64_t env = 1, tb = 1;
  for (int k = 0; k <= L; ++k) env = std::max<int64_t>(env, x->ranks[k] * y->ranks[k]);
  for (int k = 0; k < L; ++k) {
    tb = std::max<int64_t>(tb, x->ranks[k] * (int64_t)x->d[k] * y->ranks[k + 1]);
    tb = std::max<int64_t>(tb, y->ranks[k] * (int64_t)x->d[k] * x->ranks[k + 1]);
  }
  const int c = env_segment(L);
  const int ncp = (L + c - 1) / c;
  double* CP = static_cast<double*>(ws);   // checkpoints: E^L at sites 0, c, 2c, ... (env each)
  double* SEG = CP + (int64_t)ncp * env;   // the current segment's left environments
  double* ER = SEG + (int64_t)c * env;
  double* ER2 = ER + env;
  double* T1 = ER2 + env;
  double* T2 = T1 + tb;
  double* T3 = T2 + tb;
  // E^L_{k+1} from E^L_k (both FP64, rx x ry row-major)
  auto left_step = [&](int k, const double* El, double* Eout) -> int {
    const int rx0 = (int)x->ranks[k], rx1 = (int)x->ranks[k + 1];
    const int ry0 = (int)y->ranks[k], ry1 = (int)y->ranks[k + 1], d = x->d[k];
    const TX* X = static_cast<const TX*>(x->cores[k]);
    const TY* Y = static_cast<const TY*>(y->cores[k]);
    TT_TRY((gemm<double, TY, double>(s, rx0, d * ry1, ry0, 1.0, El, ry0, 1, Y, (int64_t)d * ry1, 1, 0.0, T1,
                                     (int64_t)d * ry1, 1)));
    return gemm<TX, double, double>(s, rx1, ry1, rx0 * d, 1.0, X, 1, rx1, T1, ry1, 1, 0.0, Eout, ry1, 1);
  };
  // forward: checkpoints only (the segment buffer holds the running environment)
  set_scalar_kernel<<<1, 1, 0, s>>>(CP, 1.0);
  TT_LAUNCH_CHECK();
  {
    double* run = CP;
    for (int k = 0; k < L - 1; ++k) {
      const bool cp = (k + 1) % c == 0;
      double* dst = cp ? CP + (int64_t)((k + 1) / c) * env : SEG + (int64_t)((k + 1) & 1) * env;
      TT_TRY(left_step(k, run, dst));
      run = dst;
    }
  }
  set_scalar_kernel<<<1, 1, 0, s>>>(ER, 1.0);
  TT_LAUNCH_CHECK();
  for (int seg = ncp - 1; seg >= 0; --seg) {
    const int k0 = seg * c, k1 = std::min(L, k0 + c);
    // E^L_{k0} .. E^L_{k1 - 1} of this segment into SEG[0 .. k1 - k0)
    TT_CUDA_CHECK(cudaMemcpyAsync(SEG, CP + (int64_t)seg * env,
                                  (size_t)x->ranks[k0] * y->ranks[k0] * sizeof(double), cudaMemcpyDeviceToDevice,
                                  s));
    for (int k = k0; k + 1 < k1; ++k) TT_TRY(left_step(k, SEG + (int64_t)(k - k0) * env, SEG + (int64_t)(k + 1 - k0) * env));
    for (int k = k1 - 1; k >= k0; --k) {
      const int rx0 = (int)x->ranks[k], rx1 = (int)x->ranks[k + 1];
      const int ry0 = (int)y->ranks[k], ry1 = (int)y->ranks[k + 1], d = x->d[k];
      const TX* X = static_cast<const TX*>(x->cores[k]);
      const TY* Y = static_cast<const TY*>(y->cores[k]);
      const double* El = SEG + (int64_t)(k - k0) * env;
      if (dx && dx->cores[k]) {
        // T1 = E^L Y ; dX' ((rx0 d) x rx1) += dout T1' ((rx0 d) x ry1) (E^R)^T (ry1 x rx1)
        TT_TRY((gemm<double, TY, double>(s, rx0, d * ry1, ry0, 1.0, El, ry0, 1, Y, (int64_t)d * ry1, 1,
                                         0.0, T1, (int64_t)d * ry1, 1)));
        TT_TRY((gemm<double, double, TX>(s, rx0 * d, rx1, ry1, dout, T1, ry1, 1, ER, 1, ry1, 1.0,
                                         static_cast<TX*>(dx->cores[k]), rx1, 1)));
      }
      if (dy && dy->cores[k]) {
        // T2 = (E^L)^T X  (ry0 x d rx1) ; dY' ((ry0 d) x ry1) += dout T2' ((ry0 d) x rx1) E^R
        TT_TRY((gemm<double, TX, double>(s, ry0, d * rx1, rx0, 1.0, El, 1, ry0, X, (int64_t)d * rx1, 1,
                                         0.0, T2, (int64_t)d * rx1, 1)));
        TT_TRY((gemm<double, double, TY>(s, ry0 * d, ry1, rx1, dout, T2, rx1, 1, ER, ry1, 1, 1.0,
                                         static_cast<TY*>(dy->cores[k]), ry1, 1)));
      }
      if (k > 0) {
        // T3 ((rx0 d) x ry1) = X' E^R ; E^R_new (rx0 x ry0) = T3'' (rx0 x d ry1) Y''^T
        TT_TRY((gemm<TX, double, double>(s, rx0 * d, ry1, rx1, 1.0, X, rx1, 1, ER, ry1, 1, 0.0, T3, ry1, 1)));
        TT_TRY((gemm<double, TY, double>(s, rx0, ry0, d * ry1, 1.0, T3, (int64_t)d * ry1, 1, Y, 1,
                                         (int64_t)d * ry1, 0.0, ER2, ry0, 1)));
        std::swap(ER, ER2);
      }
    }
  }
  return TT_OK;
}

// ------------------------------------------------------------------ eval
// Samples per CTA of the staged kernels: 128, or 64 when that keeps more warps resident (the
// row buffers of S samples and the staged core share the SM's 227 KB of shared memory; the
// kernels are bound by shared-memory latency, which more resident warps hide).
inline int staged_samples(size_t per_sample_bytes, size_t fixed_bytes) {
  auto warps = [&](int S) {
    const size_t b = per_sample_bytes * S + fixed_bytes + 1024;
    const int ctas = (int)std::min<size_t>(std::min<size_t>(227 * 1024 / b, 32), 2048 / S);
    return ctas * S / 32;
  };
  return warps(64) > warps(128) ? 64 : 128;
}

template <typename T>
int eval_impl(const tt_train* x, const uint8_t* digits, int64_t n, void* values, cudaStream_t s,
              unsigned* status_dev) {
  if (n == 0) return TT_OK;
  EvalParams<T> P;
  P.L = x->L;
  P.rmax = 1;
  for (int k = 0; k < x->L; ++k) {
    P.g[k] = static_cast<const T*>(x->cores[k]);
    P.d[k] = x->d[k];
    P.r[k] = (int)x->ranks[k];
    P.rmax = std::max<int>(P.rmax, (int)x->ranks[k]);
  }
  P.r[x->L] = (int)x->ranks[x->L];
  // staged form: rows of 2 x rmax x S values, the largest padded core and the digits
  {
    int stage = 1;
    for (int k = 0; k < x->L; ++k)
      stage = std::max(stage, P.r[k] * P.d[k] * eval_row_pad<T>(P.r[k + 1]));
    static std::atomic<int> configured_s[2] = {{-1}, {-1}};
    int dev = 0;
    TT_CUDA_CHECK(cudaGetDevice(&dev));
    const int which = sizeof(T) == 8 ? 0 : 1;
    if (configured_s[which] != dev) {
      TT_CUDA_CHECK(cudaFuncSetAttribute(eval_staged_kernel<T, 16, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 110 * 1024));
      if constexpr (sizeof(T) == 4)
        TT_CUDA_CHECK(cudaFuncSetAttribute(eval_staged_kernel<T, 64, true>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, 110 * 1024));
      configured_s[which] = dev;
    }
    if constexpr (sizeof(T) == 4) {
      // one pass per site, row vector updated in place
      constexpr int JB = 64;
      if (P.rmax <= JB) {
        const int SS = staged_samples((size_t)P.rmax * sizeof(T) + x->L, (stage + JB) * sizeof(T) + 16);
        const size_t bytes = ((size_t)P.rmax * SS + stage + JB) * sizeof(T) + (size_t)SS * x->L + 16;
        if (bytes <= 110 * 1024) {
          const long long blocks = ceil_div(n, SS);
          if (blocks > 0x7fffffffLL) return fail(TT_ERR_UNSUPPORTED, "tt_eval: too many samples");
          eval_staged_kernel<T, JB, true><<<(unsigned)blocks, SS, bytes, s>>>(P, digits, n, static_cast<T*>(values),
                                                                               status_dev, stage);
          TT_LAUNCH_CHECK();
          return TT_OK;
        }
      }
    }
    constexpr int JB = 16;
    const int SS = staged_samples(2 * (size_t)P.rmax * sizeof(T) + x->L, (stage + JB) * sizeof(T) + 16);
    const size_t bytes = (2 * (size_t)P.rmax * SS + stage + JB) * sizeof(T) + (size_t)SS * x->L + 16;
    if (bytes <= 110 * 1024) {
      const long long blocks = ceil_div(n, SS);
      if (blocks > 0x7fffffffLL) return fail(TT_ERR_UNSUPPORTED, "tt_eval: too many samples");
      eval_staged_kernel<T, JB, false><<<(unsigned)blocks, SS, bytes, s>>>(P, digits, n, static_cast<T*>(values),
                                                                           status_dev, stage);
      TT_LAUNCH_CHECK();
      return TT_OK;
    }
  }
  int S = 128;
  auto smem_for = [&](int SS) { return 2 * (size_t)P.rmax * SS * sizeof(T); };
  while (S > 32 && smem_for(S) > 200 * 1024) S /= 2;
  if (smem_for(S) > 200 * 1024) return fail(TT_ERR_UNSUPPORTED, "tt_eval: rank too large");
  static std::atomic<int> configured[2] = {{-1}, {-1}};
  int dev = 0;
  TT_CUDA_CHECK(cudaGetDevice(&dev));
  const int which = sizeof(T) == 8 ? 0 : 1;
  if (configured[which] != dev) {
    TT_CUDA_CHECK(cudaFuncSetAttribute(eval_kernel<T, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       200 * 1024));
    configured[which] = dev;
  }
  const long long blocks = ceil_div(n, S);
  if (blocks > 0x7fffffffLL) return fail(TT_ERR_UNSUPPORTED, "tt_eval: too many samples");
  eval_kernel<T, 8><<<(unsigned)blocks, S, smem_for(S), s>>>(P, digits, n, static_cast<T*>(values),
                                                               status_dev);
  TT_LAUNCH_CHECK();
  return TT_OK;
}

// Fallback for trains whose cores do not fit the staged kernels: samples in chunks of 16384,
// FP64 prefixes and suffixes, one thread per output element and per (a, b) of a site.
constexpr int64_t kEvalBwdChunk = 16384;

size_t eval_backward_generic_bytes(const tt_train* x, int64_t n) {
  const int64_t c = std::max<int64_t>(1, std::min<int64_t>(n, kEvalBwdChunk));
  int64_t rmax = 1, gmax = 1, pre = 0;
  for (int k = 0; k <= x->L; ++k) {
    rmax = std::max<int64_t>(rmax, x->ranks[k]);
    pre += c * x->ranks[k];
  }
  for (int k = 0; k < x->L; ++k) gmax = std::max<int64_t>(gmax, x->ranks[k] * (int64_t)x->d[k] * x->ranks[k + 1]);
  return (size_t)(pre + 2 * c * rmax + gmax + 64) * sizeof(double) + 1024;
}

template <typename T>
int eval_backward_generic(const tt_train* x, const uint8_t* digits, int64_t n, const void* dvalues,
                          tt_train* dx, void* ws, cudaStream_t s) {
  const int L = x->L;
  const int64_t chunk = std::min<int64_t>(n, kEvalBwdChunk);
  int64_t rmax = 1;
  for (int k = 0; k <= L; ++k) rmax = std::max<int64_t>(rmax, x->ranks[k]);
  std::vector<int64_t> poff(L + 1);
  int64_t off = 0;
  for (int k = 0; k <= L; ++k) {
    poff[k] = off;
    off += chunk * x->ranks[k];
  }
  double* pre = static_cast<double*>(ws);
  double* sA0 = pre + off;
  double* sB0 = sA0 + chunk * rmax;
  double* acc = sB0 + chunk * rmax;
  const int TPB = 256;
  for (int64_t c0 = 0; c0 < n; c0 += chunk) {
    const int64_t cn = std::min<int64_t>(chunk, n - c0);
    const uint8_t* dg = digits + c0 * L;
    const T* w = static_cast<const T*>(dvalues) + c0;
    double* sA = sA0;
    double* sB = sB0;
    fill_ones_kernel<<<(unsigned)ceil_div(cn, TPB), TPB, 0, s>>>(pre, cn);
    TT_LAUNCH_CHECK();
    for (int k = 0; k < L - 1; ++k) {
      const int r0 = (int)x->ranks[k], r1 = (int)x->ranks[k + 1];
      eval_step_kernel<T><<<(unsigned)ceil_div(cn * r1, TPB), TPB, 0, s>>>(
          static_cast<const T*>(x->cores[k]), r0, x->d[k], r1, dg, L, k, cn, pre + poff[k],
          pre + poff[k + 1], false);
      TT_LAUNCH_CHECK();
    }
    fill_ones_kernel<<<(unsigned)ceil_div(cn, TPB), TPB, 0, s>>>(sA, cn);
    TT_LAUNCH_CHECK();
    for (int k = L - 1; k >= 0; --k) {
      const int r0 = (int)x->ranks[k], r1 = (int)x->ranks[k + 1], d = x->d[k];
      if (dx->cores[k]) {
        const int64_t g = (int64_t)r0 * d * r1;
        TT_CUDA_CHECK(cudaMemsetAsync(acc, 0, g * sizeof(double), s));
        dim3 grid((unsigned)std::min<int64_t>(std::max<int64_t>(1, cn / 256), 256), (unsigned)r0);
        eval_bwd_site_kernel<T><<<grid, 128, 0, s>>>(pre + poff[k], sA, w, dg, L, k, cn, r0, d, r1, acc);
        TT_LAUNCH_CHECK();
        add_into_kernel<T><<<(unsigned)ceil_div(g, TPB), TPB, 0, s>>>(acc, g, static_cast<T*>(dx->cores[k]));
        TT_LAUNCH_CHECK();
      }
      if (k > 0) {
        eval_step_kernel<T><<<(unsigned)ceil_div(cn * r0, TPB), TPB, 0, s>>>(
            static_cast<const T*>(x->cores[k]), r0, d, r1, dg, L, k, cn, sA, sB, true);
        TT_LAUNCH_CHECK();
        std::swap(sA, sB);
      }
    }
  }
  return TT_OK;
}

// Staged path: shared memory of eval_states_kernel (two row buffers of S samples, the largest
// staged core in either orientation, the CTA's digits).
constexpr int kStatesJB = 16;
constexpr size_t kStatesSmemMax = 110 * 1024;
constexpr size_t kStateBudget = size_t(1) << 30;  // bytes of prefix + suffix states per chunk

template <typename T>
int states_stage_elems(const tt_train* x) {
  int stage = 1;
  for (int k = 0; k < x->L; ++k) {
    const int r0 = (int)x->ranks[k], r1 = (int)x->ranks[k + 1], d = x->d[k];
    stage = std::max(stage, std::max(r0 * d * eval_row_pad<T>(r1), r1 * d * eval_row_pad<T>(r0)));
  }
  return stage;
}

// FP32 trains of rank <= 64 take the one-pass, in-place form (one row buffer)
template <typename T>
bool states_one(const tt_train* x) {
  int rmax = 1;
  for (int k = 0; k <= x->L; ++k) rmax = std::max<int>(rmax, (int)x->ranks[k]);
  return sizeof(T) == 4 && rmax <= 64;
}

template <typename T>
int states_samples(const tt_train* x) {
  int rmax = 1;
  for (int k = 0; k <= x->L; ++k) rmax = std::max<int>(rmax, (int)x->ranks[k]);
  const int nbuf = states_one<T>(x) ? 1 : 2, jb = states_one<T>(x) ? 64 : kStatesJB;
  return staged_samples(nbuf * (size_t)rmax * sizeof(T) + x->L, (states_stage_elems<T>(x) + jb) * sizeof(T) + 16);
}

template <typename T>
size_t states_smem(const tt_train* x, int S) {
  int rmax = 1;
  for (int k = 0; k <= x->L; ++k) rmax = std::max<int>(rmax, (int)x->ranks[k]);
  const int nbuf = states_one<T>(x) ? 1 : 2, jb = states_one<T>(x) ? 64 : kStatesJB;
  return (nbuf * (size_t)rmax * S + states_stage_elems<T>(x) + jb) * sizeof(T) + (size_t)S * x->L + 16;
}

// samples per chunk of the state store, and the store's elements per sample
template <typename T>
int64_t states_chunk(const tt_train* x, int64_t n, int64_t* per_sample) {
  int64_t per = 0;
  for (int k = 0; k < x->L; ++k) per += x->ranks[k] + x->ranks[k + 1];
  if (per_sample) *per_sample = per;
  int64_t c = (int64_t)(kStateBudget / ((size_t)per * sizeof(T))) & ~int64_t(127);
  c = std::max<int64_t>(128, std::min<int64_t>(c, 65536));
  return std::max<int64_t>(1, std::min<int64_t>(c, n));
}

template <typename T>
size_t eval_backward_staged_bytes(const tt_train* x, int64_t n) {
  int64_t per = 0;
  const int64_t C = states_chunk<T>(x, n, &per);
  int64_t g = 0;
  for (int k = 0; k < x->L; ++k) g += x->ranks[k] * (int64_t)x->d[k] * x->ranks[k + 1];
  return ((size_t)C * per * sizeof(T) + 255) / 256 * 256 + (size_t)g * sizeof(double) + 1024;
}

template <typename T>
bool eval_backward_staged_fits(const tt_train* x) {
  return states_smem<T>(x, 64) <= kStatesSmemMax;
}

size_t eval_backward_workspace_bytes(const tt_train* x, int64_t n) {
  if (x->dtype == TT_F64)
    return eval_backward_staged_fits<double>(x) ? eval_backward_staged_bytes<double>(x, n)
                                                : eval_backward_generic_bytes(x, n);
  return eval_backward_staged_fits<float>(x) ? eval_backward_staged_bytes<float>(x, n)
                                             : eval_backward_generic_bytes(x, n);
}

template <typename T>
int eval_backward_impl(const tt_train* x, const uint8_t* digits, int64_t n, const void* dvalues,
                       tt_train* dx, void* ws, size_t ws_bytes, cudaStream_t s) {
  if (n == 0) return TT_OK;
  if (ws_bytes < eval_backward_workspace_bytes(x, n))
    return fail(TT_ERR_WORKSPACE, "tt_eval_backward: workspace too small");
  if (!eval_backward_staged_fits<T>(x)) return eval_backward_generic<T>(x, digits, n, dvalues, dx, ws, s);
  const int L = x->L;
  EvalParams<T> P;
  P.L = L;
  P.rmax = 1;
  SiteMask want;
  bool any = false;
  for (int k = 0; k < L; ++k) {
    P.g[k] = static_cast<const T*>(x->cores[k]);
    P.d[k] = x->d[k];
    P.r[k] = (int)x->ranks[k];
    P.rmax = std::max<int>(P.rmax, (int)x->ranks[k]);
    want.on[k] = dx->cores[k] != nullptr;
    any = any || want.on[k];
  }
  P.r[L] = (int)x->ranks[L];
  if (!any) return TT_OK;
  int64_t per = 0;
  const int64_t C = states_chunk<T>(x, n, &per);
  T* states = static_cast<T*>(ws);
  double* acc = reinterpret_cast<double*>(static_cast<char*>(ws) + ((size_t)C * per * sizeof(T) + 255) / 256 * 256);
  int64_t g = 0, zdim = 0;
  constexpr int DG = sizeof(T) == 4 ? 2 : 1;
  int tiles = 1;
  for (int k = 0; k < L; ++k) {
    g += x->ranks[k] * (int64_t)x->d[k] * x->ranks[k + 1];
    zdim += (x->d[k] + DG - 1) / DG;
    tiles = std::max<int>(tiles, (int)(ceil_div(x->ranks[k], kAccTile) * ceil_div(x->ranks[k + 1], kAccTile)));
  }
  if (zdim > 65535 || tiles > 65535) return fail(TT_ERR_UNSUPPORTED, "tt_eval_backward: train too large");
  TT_CUDA_CHECK(cudaMemsetAsync(acc, 0, (size_t)g * sizeof(double), s));
  int S = states_samples<T>(x);
  if (states_smem<T>(x, S) > kStatesSmemMax) S = 64;
  const size_t smem = states_smem<T>(x, S);
  const int stage = states_stage_elems<T>(x);
  static std::atomic<int> configured[2] = {{-1}, {-1}};
  int dev = 0;
  TT_CUDA_CHECK(cudaGetDevice(&dev));
  const int which = sizeof(T) == 8 ? 0 : 1;
  if (configured[which] != dev) {
    TT_CUDA_CHECK(cudaFuncSetAttribute(eval_states_kernel<T, kStatesJB, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStatesSmemMax));
    if constexpr (sizeof(T) == 4)
      TT_CUDA_CHECK(cudaFuncSetAttribute(eval_states_kernel<T, 64, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kStatesSmemMax));
    configured[which] = dev;
  }
  // slices of at most 2048 samples (the FP32 sums of a slice stay short) and enough CTAs to fill the GPU
  const int64_t slice_target = std::max<int64_t>(256, std::min<int64_t>(2048, C / std::max<int64_t>(1, ceil_div(4 * num_sms(), zdim * tiles))));
  for (int64_t c0 = 0; c0 < n; c0 += C) {
    const int64_t cn = std::min<int64_t>(C, n - c0);
    const uint8_t* dg = digits + c0 * L;
    const T* w = static_cast<const T*>(dvalues) + c0;
    if constexpr (sizeof(T) == 4) {
      if (states_one<T>(x))
        eval_states_kernel<T, 64, true><<<dim3((unsigned)ceil_div(cn, S), 2), S, smem, s>>>(P, dg, cn, states, C,
                                                                                          stage);
      else
        eval_states_kernel<T, kStatesJB, false><<<dim3((unsigned)ceil_div(cn, S), 2), S, smem, s>>>(
            P, dg, cn, states, C, stage);
    } else {
      eval_states_kernel<T, kStatesJB, false><<<dim3((unsigned)ceil_div(cn, S), 2), S, smem, s>>>(P, dg, cn, states,
                                                                                                  C, stage);
    }
    TT_LAUNCH_CHECK();
    const int64_t slice = (std::min<int64_t>(slice_target, cn) + kAccK - 1) / kAccK * kAccK;
    const dim3 grid((unsigned)ceil_div(cn, slice), (unsigned)tiles, (unsigned)zdim);
    eval_bwd_accum_kernel<T, DG><<<grid, 128, 0, s>>>(P, want, dg, w, cn, states, C, slice, acc);
    TT_LAUNCH_CHECK();
  }
  const int TPB = 256;
  int64_t off = 0;
  for (int k = 0; k < L; ++k) {
    const int64_t gk = x->ranks[k] * (int64_t)x->d[k] * x->ranks[k + 1];
    if (want.on[k]) {
      add_into_kernel<T><<<(unsigned)ceil_div(gk, TPB), TPB, 0, s>>>(acc + off, gk, static_cast<T*>(dx->cores[k]));
      TT_LAUNCH_CHECK();
    }
    off += gk;
  }
  return TT_OK;
}

template int inner_impl<double, double>(const tt_train*, const tt_train*, double*, void*, size_t, cudaStream_t);
template int inner_impl<float, float>(const tt_train*, const tt_train*, double*, void*, size_t, cudaStream_t);
template int inner_backward_impl<double, double>(const tt_train*, const tt_train*, double, tt_train*,
                                                 tt_train*, void*, size_t, cudaStream_t);
template int inner_backward_impl<float, float>(const tt_train*, const tt_train*, double, tt_train*,
                                               tt_train*, void*, size_t, cudaStream_t);
template int eval_impl<double>(const tt_train*, const uint8_t*, int64_t, void*, cudaStream_t, unsigned*);
template int eval_impl<float>(const tt_train*, const uint8_t*, int64_t, void*, cudaStream_t, unsigned*);
template int eval_backward_impl<double>(const tt_train*, const uint8_t*, int64_t, const void*, tt_train*,
                                        void*, size_t, cudaStream_t);
template int eval_backward_impl<float>(const tt_train*, const uint8_t*, int64_t, const void*, tt_train*,
                                       void*, size_t, cudaStream_t);

}  // namespace tt
