// Householder panel factorisation and block-reflector application for the rounding sweeps.
//
// Panel (qr_panel_fast): FP64 arithmetic, one thread-block cluster barrier per column.
// The panel rows are split over the cluster's CTAs (each keeps its rows of the panel in
// shared memory, column-major with an odd leading dimension).  For column c every CTA
// forms, over its own rows below the diagonal, the dot products of the still unscaled
// column x = A[:, c] with every panel column t:
//     S_t = sum_{l > c} x_l A[l, t]          (t = c: the squared norm below the diagonal)
// and the owner of row c publishes that row.  After ONE cluster barrier every CTA has
// what the Householder step needs:
//     beta = -sign(alpha) sqrt(alpha^2 + S_c),  tau = (beta - alpha) / beta,
//     v = [1; x / (alpha - beta)],  d_t = A[c, t] + S_t / (alpha - beta) = v^T a_t,
// where for t < c (a previous reflector v_t) d_t = v_t^T v, the entries of column c of T:
// T[:c, c] = -tau T[:c, :c] d[:c].  The reduction and the scaling are deferred until after
// the sums, so one exchange per column replaces the usual two (norm, then dot products).
// Threads are mapped as (row group, column): lane t of a row group owns column t, so a dot
// product is one FMA per row and thread and the cross-thread reduction is a short sum over
// row groups - on GB300 every FP64 instruction of a warp holds the SM's FP64 pipe for 16
// cycles, so reduction trees over many accumulators cost more than the dot products.
//
// Block reflector (apply_block_reflector): W1 = V^T X, W2 = op(T) W1, X -= V W2 in one
// launch, one CTA per block of columns of X.
#include <cooperative_groups.h>

#include <type_traits>

#include "tt_panel.cuh"

namespace cg = cooperative_groups;

namespace tt {

namespace {

constexpr int PT = 256;              // threads of the panel kernel
constexpr int kPanelCluster = 8;     // CTAs of a cluster panel
constexpr size_t kPanelSmemMax = 200 * 1024;

template <int NB>
__host__ __device__ constexpr int gram_pairs() {
  return NB * (NB + 1) / 2;
}

template <int CS>
__device__ __forceinline__ void panel_sync() {
  if constexpr (CS > 1) cluster_sync_all();
  else __syncthreads();
}

template <int CS>
__device__ __forceinline__ double panel_load(const double* p, int rank) {
  if constexpr (CS > 1) return dsmem_load(p, rank);
  else {
    (void)rank;
    return *p;
  }
}

// (s, t), s <= t, of Gram pair index q = t (t + 1) / 2 + s
__device__ __forceinline__ void pair_of(int q, int& s, int& t) {
  int tt = (int)((sqrtf(8.0f * (float)q + 1.0f) - 1.0f) * 0.5f);
  while ((tt + 1) * (tt + 2) / 2 <= q) ++tt;
  while (tt * (tt + 1) / 2 > q) --tt;
  t = tt;
  s = q - tt * (tt + 1) / 2;
}

// The panel of jb columns at (j0, j0) of A, rows [j0, m): local rows l in [0, mr) split as
// [rank * chunk, (rank + 1) * chunk) over CS CTAs.  ldp = chunk | 1.
template <typename TIO, int NB, int CS>
__device__ __forceinline__ void panel_fast_body(TIO* __restrict__ A, int lda, int m, int j0, int jb,
                                                TIO* __restrict__ tau, double* __restrict__ Tm, int ldt,
                                                TIO* __restrict__ Vb, int ldv, int chunk, int rank) {
  constexpr int NRG = PT / NB;  // row groups
  constexpr bool kRound = std::is_same<TIO, float>::value;
  extern __shared__ double P[];  // P[t * ldp + (l - lo)]
  __shared__ double red[NRG][NB];
  __shared__ double slot[2][NB];     // this CTA's partial S_t of the last two columns
  __shared__ double rowslot[2][NB];  // row c of the panel (owner CTA)
  __shared__ double Ts[NB][NB + 1];
  __shared__ double sh_d[NB];
  __shared__ double sh_tau, sh_scal;
  __shared__ double gpart[kRound ? gram_pairs<NB>() : 1];
  const int tid = threadIdx.x, t = tid % NB, g = tid / NB;
  const int mr = m - j0;
  const int ldp = chunk | 1;
  const int lo = min(mr, rank * chunk), hi = min(mr, (rank + 1) * chunk);
  for (int c = 0; c < jb; ++c) {
    const TIO* src = A + (int64_t)(j0 + c) * lda + j0;
    for (int l = lo + tid; l < hi; l += PT) P[c * ldp + (l - lo)] = (double)src[l];
  }
  for (int e = tid; e < NB * (NB + 1); e += PT) (&Ts[0][0])[e] = 0.0;
  __syncthreads();

  for (int c = 0; c < jb; ++c) {
    const int b = c & 1;
    const int owner = c / chunk;
    const bool own = rank == owner;
    const int r0 = max(lo, c + 1);
    // ---- 1. partial S_t over own rows below the diagonal; the owner publishes row c
    double acc = 0.0;
    if (t < jb) {
      const double* pc = P + c * ldp - lo;
      const double* pt = P + t * ldp - lo;
      for (int l = r0 + g; l < hi; l += NRG) acc = fma(pc[l], pt[l], acc);
    }
    // a warp holds 32 / NB row groups of the same columns: fold them first (one shuffle
    // level for NB = 16), then sum the warps' partials
    static_assert(NB == 16 || NB == 32, "panel width");
    if constexpr (NB == 16) acc += __shfl_xor_sync(0xffffffffu, acc, 16);
    constexpr int NWP = NRG * NB / 32;  // warps
    if (NB == 32 || (tid & 16) == 0) red[NB == 16 ? g >> 1 : g][t] = acc;
    if (own && g == 0) rowslot[b][t] = t < jb ? P[t * ldp + (c - lo)] : 0.0;
    __syncthreads();
    if (tid < NB) {
      double sum = 0.0;
#pragma unroll
      for (int q = 0; q < NWP; ++q) sum += red[q][tid];
      slot[b][tid] = sum;
    }
    panel_sync<CS>();
    // ---- 2. totals, the reflector, d_t, column c of T; the owner finishes row c
    if (tid < 32) {
      const int lane = tid;
      double S = 0.0, rv = 0.0;
      if (lane < jb) {
        double part[CS];
#pragma unroll
        for (int r = 0; r < CS; ++r) part[r] = panel_load<CS>(&slot[b][lane], r);
        rv = panel_load<CS>(&rowslot[b][lane], owner);
#pragma unroll
        for (int r = 0; r < CS; ++r) S += part[r];
      }
      const double ss = __shfl_sync(0xffffffffu, S, c);
      const double alpha = __shfl_sync(0xffffffffu, rv, c);
      double tc = 0.0, sc = 1.0, beta = alpha;
      if (ss != 0.0) {
        beta = -copysign(sqrt(alpha * alpha + ss), alpha);
        // tau = (beta - alpha) / beta and the scale 1 / (alpha - beta) from one division:
        // with e = alpha - beta and q = 1 / (beta e), tau = -e^2 q, scale = beta q
        const double e = alpha - beta;
        const double q = 1.0 / (beta * e);
        tc = -(e * e) * q;
        sc = beta * q;
      }
      const double dd = rv + sc * S;
      if (lane < jb) sh_d[lane] = dd;
      __syncwarp();
      if (lane < c) {
        double v = 0.0;
        for (int q = lane; q < c; ++q) v = fma(Ts[lane][q], sh_d[q], v);
        Ts[lane][c] = -tc * v;
      }
      if (lane == 0) {
        Ts[c][c] = tc;
        sh_tau = tc;
        sh_scal = sc;
      }
      if (own) {
        if (lane == c) P[c * ldp + (c - lo)] = beta;
        else if (lane > c && lane < jb) P[lane * ldp + (c - lo)] = rv - tc * dd;
      }
    }
    __syncthreads();
    // ---- 3. own rows below the diagonal: v_l = x_l / (alpha - beta), a_t -= tau d_t v
    const double sc = sh_scal;
    const double f = (t > c && t < jb) ? sh_tau * sh_d[t] * sc : 0.0;
    for (int base = r0; base < hi; base += NRG) {
      const int l = base + g;
      const bool in = l < hi;
      const double x = in ? P[c * ldp + (l - lo)] : 0.0;
      __syncwarp();  // every lane has read x before lane c overwrites it
      if (in) {
        if (t == c) P[c * ldp + (l - lo)] = x * sc;
        else if (t > c && t < jb) P[t * ldp + (l - lo)] = fma(-f, x, P[t * ldp + (l - lo)]);
      }
    }
    __syncthreads();
  }

  // ---- write-back: R and the reflectors in place, the explicit V; T and tau
  for (int tc = 0; tc < jb; ++tc) {
    const int jc = j0 + tc;
    TIO* dstA = A + (int64_t)jc * lda + j0;
    TIO* dstV = Vb + (int64_t)jc * ldv + j0;
    for (int l = lo + tid; l < hi; l += PT) {
      const double v = P[tc * ldp + (l - lo)];
      dstA[l] = (TIO)v;
      dstV[l] = (l < tc) ? TIO(0) : (l == tc ? TIO(1) : (TIO)v);
    }
  }
  if constexpr (!kRound) {
    if (rank == 0) {
      for (int e = tid; e < jb * jb; e += PT) {
        const int r = e % jb, cc = e / jb;
        Tm[r + (int64_t)cc * ldt] = Ts[r][cc];
      }
      if (tid < jb) tau[j0 + tid] = Ts[tid][tid];
    }
    if constexpr (CS > 1) cluster_sync_all();  // no CTA leaves while a peer may read its slots
  } else {
    // ---- mixed form: G = V'^T V' of the FP32-rounded reflectors (compensated FP32 sums of
    // exact products), tau'_t = 2 / G_tt, and T' by the same recurrence in FP64
    const int npairs = jb * (jb + 1) / 2;
    for (int q = tid; q < npairs; q += PT) {
      int s, u;
      pair_of(q, s, u);  // s <= u; v_s[l] v_u[l] is nonzero only for l >= u
      float hi32 = 0.0f, lo32 = 0.0f;
      const int l0 = max(lo, u);
      for (int l = l0; l < hi; ++l) {
        const float a = (l == s) ? 1.0f : (float)P[s * ldp + (l - lo)];
        const float bb = (l == u) ? 1.0f : (float)P[u * ldp + (l - lo)];
        const float p = __fmul_rn(a, bb);
        const float e = __fmaf_rn(a, bb, -p);
        const float ssum = __fadd_rn(hi32, p);
        const float z = __fsub_rn(ssum, hi32);
        const float err = __fadd_rn(__fsub_rn(hi32, __fsub_rn(ssum, z)), __fsub_rn(p, z));
        hi32 = ssum;
        lo32 = __fadd_rn(lo32, __fadd_rn(err, e));
      }
      gpart[q] = (double)hi32 + (double)lo32;
    }
    panel_sync<CS>();
    if (rank == 0) {
      __shared__ double G[NB][NB + 1];
      for (int q = tid; q < npairs; q += PT) {
        int s, u;
        pair_of(q, s, u);
        double sum = 0.0;
        for (int r = 0; r < CS; ++r) sum += panel_load<CS>(&gpart[q], r);
        G[s][u] = sum;
      }
      __syncthreads();
      if (tid < 32) {
        const int lane = tid;
        for (int c = 0; c < jb; ++c) {
          const double t_old = Ts[c][c];
          const double tnew = (t_old == 0.0 || G[c][c] == 0.0) ? 0.0 : 2.0 / G[c][c];
          __syncwarp();
          if (lane < c) {
            double v = 0.0;
            for (int q = lane; q < c; ++q) v = fma(Ts[lane][q], G[q][c], v);
            Ts[lane][c] = -tnew * v;
          }
          __syncwarp();
          if (lane == 0) Ts[c][c] = tnew;
          __syncwarp();
        }
      }
      __syncthreads();
      for (int e = tid; e < jb * jb; e += PT) {
        const int r = e % jb, cc = e / jb;
        Tm[r + (int64_t)cc * ldt] = r <= cc ? Ts[r][cc] : 0.0;
      }
      if (tid < jb) tau[j0 + tid] = (TIO)Ts[tid][tid];
    }
    if constexpr (CS > 1) cluster_sync_all();
  }
}

template <typename TIO, int NB, int CS>
__global__ void __launch_bounds__(PT) panel_fast_kernel(TIO* A, int lda, int m, int j0, int jb, TIO* tau,
                                                        double* Tm, int ldt, TIO* Vb, int ldv, int chunk) {
  int rank = 0;
  if constexpr (CS > 1) rank = (int)cg::this_cluster().block_rank();
  panel_fast_body<TIO, NB, CS>(A, lda, m, j0, jb, tau, Tm, ldt, Vb, ldv, chunk, rank);
}

// one job per cluster of CS CTAs (CS = 1: per CTA)
template <typename TIO, int NB, int CS>
__global__ void __launch_bounds__(PT) panel_fast_batched_kernel(const PanelJob* __restrict__ jobs, int j0, int nb) {
  const PanelJob J = jobs[blockIdx.x / CS];
  const int p = min(J.m, J.n);
  if (j0 >= p) return;  // uniform over the cluster: no CTA reaches a cluster barrier
  int rank = 0;
  if constexpr (CS > 1) rank = (int)cg::this_cluster().block_rank();
  const int jb = min(nb, p - j0);
  const int chunk = (J.m - j0 + CS - 1) / CS;
  panel_fast_body<TIO, NB, CS>(static_cast<TIO*>(J.A), J.lda, J.m, j0, jb, static_cast<TIO*>(J.tau),
                               J.Tm + (int64_t)(j0 / nb) * nb * nb, nb, static_cast<TIO*>(J.Vb), J.ldv, chunk,
                               rank);
}

size_t panel_smem(int nb, int chunk) { return (size_t)nb * (size_t)(chunk | 1) * sizeof(double); }

template <typename K>
int allow_smem(K kernel, size_t bytes) {
  TT_CUDA_CHECK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return TT_OK;
}

template <typename TIO, int NB, int CS>
int launch_panel(cudaStream_t s, TIO* A, int lda, int m, int j0, int jb, TIO* tau, double* Tm, int ldt, TIO* Vb,
                 int ldv, int chunk) {
  static std::atomic<int> configured{-1};
  int dev = 0;
  TT_CUDA_CHECK(cudaGetDevice(&dev));
  if (configured != dev) {
    TT_TRY(allow_smem(panel_fast_kernel<TIO, NB, CS>, kPanelSmemMax));
    configured = dev;
  }
  const size_t smem = panel_smem(NB, chunk);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CS);
  cfg.blockDim = dim3(PT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = CS > 1 ? 1 : 0;
  TT_CUDA_CHECK(cudaLaunchKernelEx(&cfg, panel_fast_kernel<TIO, NB, CS>, A, lda, m, j0, jb, tau, Tm, ldt, Vb, ldv,
                                   chunk));
  note_launch();
  return TT_OK;
}

template <typename TIO, int NB>
int panel_dispatch(cudaStream_t s, TIO* A, int lda, int m, int j0, int jb, TIO* tau, double* Tm, int ldt, TIO* Vb,
                   int ldv) {
  const int mr = m - j0;
  if (mr >= 256) {
    const int chunk = (mr + kPanelCluster - 1) / kPanelCluster;
    if (panel_smem(NB, chunk) > kPanelSmemMax) return fail(TT_ERR_UNSUPPORTED, "qr panel: too many rows");
    return launch_panel<TIO, NB, kPanelCluster>(s, A, lda, m, j0, jb, tau, Tm, ldt, Vb, ldv, chunk);
  }
  return launch_panel<TIO, NB, 1>(s, A, lda, m, j0, jb, tau, Tm, ldt, Vb, ldv, mr);
}

// ------------------------------------------------------------------ block reflector
constexpr int RT = 256;   // threads
constexpr int RCH = 128;  // rows of V staged per chunk

// X[:, c0 .. c0 + RNC) <- (I - V op(T) V^T) X[:, ...]; RNC columns of X per CTA
template <typename T, int NB, int RNC>
__device__ __forceinline__ void reflector_body(const T* __restrict__ V, int ldv, int mr, int jb,
                                               const double* __restrict__ Tm, int ldt, bool transpose_t,
                                               T* __restrict__ X, int ldx, int nc, int c0) {
  constexpr bool kMixed = std::is_same<T, float>::value;
  constexpr int NO = NB * RNC;      // outputs of W1
  constexpr int NG = RT / NO;       // row groups of the W1 reduction
  static_assert(NG * NO == RT, "reflector layout");
  __shared__ T Vs[RCH][NB + 1];
  __shared__ T Xs[RCH][RNC];
  __shared__ double wred[NG][NO];
  __shared__ double W2[NB][RNC];
  __shared__ float W2h[NB][RNC], W2l[NB][RNC];
  const int tid = threadIdx.x;
  const int o = tid % NO, g = tid / NO;
  const int q = o / RNC, j = o % RNC;
  const int ncol = min(RNC, nc - c0);
  // ---- W1 = V^T X over row chunks staged in shared memory
  double acc = 0.0;
  float ah = 0.0f, al = 0.0f;
  for (int l0 = 0; l0 < mr; l0 += RCH) {
    const int rows = min(RCH, mr - l0);
    {
      // all of a thread's loads of the chunk are issued before its stores
      constexpr int UV = RCH * NB / RT, UX = (RCH * RNC + RT - 1) / RT;
      T vv[UV], xv[UX];
#pragma unroll
      for (int u = 0; u < UV; ++u) {
        const int e = tid + u * RT, r = e % RCH, c = e / RCH;
        vv[u] = (r < rows && c < jb) ? V[(int64_t)c * ldv + l0 + r] : T(0);
      }
#pragma unroll
      for (int u = 0; u < UX; ++u) {
        const int e = tid + u * RT, r = e % RCH, c = e / RCH;
        xv[u] = (e < RCH * RNC && r < rows && c < ncol) ? X[(int64_t)(c0 + c) * ldx + l0 + r] : T(0);
      }
#pragma unroll
      for (int u = 0; u < UV; ++u) {
        const int e = tid + u * RT;
        Vs[e % RCH][e / RCH] = vv[u];
      }
#pragma unroll
      for (int u = 0; u < UX; ++u) {
        const int e = tid + u * RT;
        if (e < RCH * RNC) Xs[e % RCH][e / RCH] = xv[u];
      }
    }
    __syncthreads();
    if constexpr (kMixed) {
      for (int r = g; r < rows; r += NG) {
        const float a = Vs[r][q], bb = Xs[r][j];
        const float p = __fmul_rn(a, bb);
        const float e = __fmaf_rn(a, bb, -p);
        const float s = __fadd_rn(ah, p);
        const float z = __fsub_rn(s, ah);
        const float err = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, z)), __fsub_rn(p, z));
        ah = s;
        al = __fadd_rn(al, __fadd_rn(err, e));
      }
    } else {
      for (int r = g; r < rows; r += NG) acc = fma((double)Vs[r][q], (double)Xs[r][j], acc);
    }
    __syncthreads();
  }
  if constexpr (kMixed) acc = (double)ah + (double)al;
  wred[g][o] = acc;
  __syncthreads();
  // ---- W2 = op(T) W1 (FP64)
  __shared__ double W1s[NB][RNC];
  if (tid < NO) {
    double sum = 0.0;
#pragma unroll
    for (int gg = 0; gg < NG; ++gg) sum += wred[gg][tid];
    W1s[tid / RNC][tid % RNC] = sum;
  }
  __syncthreads();
  if (tid < NO) {
    double v = 0.0;
    if (q < jb) {
      if (transpose_t) {  // (T^T w)_q = sum_{r <= q} T[r, q] w_r
        for (int r = 0; r <= q; ++r) v = fma(Tm[r + (int64_t)q * ldt], W1s[r][j], v);
      } else {  // (T w)_q = sum_{r >= q} T[q, r] w_r
        for (int r = q; r < jb; ++r) v = fma(Tm[q + (int64_t)r * ldt], W1s[r][j], v);
      }
    }
    W2[q][j] = v;
    if constexpr (kMixed) {
      const float h = (float)v;
      W2h[q][j] = h;
      W2l[q][j] = (float)(v - (double)h);
    }
  }
  __syncthreads();
  // ---- X -= V W2, one thread per row and all RNC columns: the jb entries of the row of V
  // are loaded together (coalesced along rows) and each feeds RNC products
  for (int l = tid; l < mr; l += RT) {
    T vr[NB];
#pragma unroll
    for (int r = 0; r < NB; ++r) vr[r] = r < jb ? V[(int64_t)r * ldv + l] : T(0);
#pragma unroll
    for (int jj = 0; jj < RNC; ++jj) {
      if (jj >= ncol) break;
      T* px = X + (int64_t)(c0 + jj) * ldx + l;
      if constexpr (kMixed) {
        float sh = 0.0f, sl = 0.0f;
#pragma unroll
        for (int r = 0; r < NB; ++r) {
          if (r < jb) {
            const float a = vr[r];
            const float wh = W2h[r][jj];
            const float p = __fmul_rn(a, wh);
            const float er = __fmaf_rn(a, wh, -p);
            const float s = __fadd_rn(sh, p);
            const float z = __fsub_rn(s, sh);
            const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, z)), __fsub_rn(p, z));
            sh = s;
            sl = __fadd_rn(sl, __fadd_rn(err, __fmaf_rn(a, W2l[r][jj], er)));
          }
        }
        *px = (float)((double)*px - ((double)sh + (double)sl));
      } else {
        double v = 0.0;
#pragma unroll
        for (int r = 0; r < NB; ++r)
          if (r < jb) v = fma((double)vr[r], W2[r][jj], v);
        *px = (T)((double)*px - v);
      }
    }
  }
}

template <typename T, int NB, int RNC>
__global__ void __launch_bounds__(RT) reflector_kernel(const T* V, int ldv, int mr, int jb, const double* Tm, int ldt,
                                                       bool transpose_t, T* X, int ldx, int nc) {
  reflector_body<T, NB, RNC>(V, ldv, mr, jb, Tm, ldt, transpose_t, X, ldx, nc, blockIdx.x * RNC);
}

}  // namespace

template <typename TIO>
int qr_panel_fast(cudaStream_t s, TIO* A, int lda, int m, int j0, int jb, int nb, TIO* tau, double* Tm, int ldt,
                  TIO* Vb, int ldv) {
  if (jb <= 0) return TT_OK;
  if (nb == 16 && jb <= 16) return panel_dispatch<TIO, 16>(s, A, lda, m, j0, jb, tau, Tm, ldt, Vb, ldv);
  if (nb == 32 && jb <= 32) return panel_dispatch<TIO, 32>(s, A, lda, m, j0, jb, tau, Tm, ldt, Vb, ldv);
  return fail(TT_ERR_UNSUPPORTED, "qr panel: width must be 16 or 32");
}

template <typename T>
int apply_block_reflector(cudaStream_t s, const T* V, int ldv, int mr, int jb, const double* Tm, int ldt,
                          bool transpose_t, T* X, int ldx, int nc) {
  if (nc <= 0 || mr <= 0 || jb <= 0) return TT_OK;
  // two columns of X per CTA, or one when that still leaves SMs idle (a CTA's time is its
  // columns' 4 mr jb multiply-adds on one SM's FP64 pipe)
  const bool one = nc <= num_sms();
  const unsigned grid = (unsigned)ceil_div(nc, one ? 1 : 2);
  if (jb <= 16) {
    if (one) reflector_kernel<T, 16, 1><<<grid, RT, 0, s>>>(V, ldv, mr, jb, Tm, ldt, transpose_t, X, ldx, nc);
    else reflector_kernel<T, 16, 2><<<grid, RT, 0, s>>>(V, ldv, mr, jb, Tm, ldt, transpose_t, X, ldx, nc);
  } else if (jb <= 32) {
    if (one) reflector_kernel<T, 32, 1><<<grid, RT, 0, s>>>(V, ldv, mr, jb, Tm, ldt, transpose_t, X, ldx, nc);
    else reflector_kernel<T, 32, 2><<<grid, RT, 0, s>>>(V, ldv, mr, jb, Tm, ldt, transpose_t, X, ldx, nc);
  } else {
    return fail(TT_ERR_UNSUPPORTED, "block reflector: width above 32");
  }
  TT_LAUNCH_CHECK();
  return TT_OK;
}

template <typename TIO>
int qr_panel_fast_batched(cudaStream_t s, int njobs, const PanelJob* d_jobs, int j0, int nb, int mr_max) {
  if (njobs <= 0 || mr_max <= 0) return TT_OK;
  // cluster size per job: the smallest power of two whose row share fits shared memory
  int cs = 1;
  while (cs < kPanelCluster && panel_smem(nb, (mr_max + cs - 1) / cs) > kPanelSmemMax) cs *= 2;
  // with few jobs, spread each job's rows over more SMs (a panel is bound by the FP64 pipe of
  // the SMs that hold it): grow the cluster while all CTAs still fit one wave and every CTA
  // keeps at least 64 rows
  while (cs < kPanelCluster && (int64_t)njobs * cs * 2 <= num_sms() && mr_max / (cs * 2) >= 64) cs *= 2;
  const int chunk = (mr_max + cs - 1) / cs;
  const size_t smem = panel_smem(nb, chunk);
  if (smem > kPanelSmemMax) return fail(TT_ERR_UNSUPPORTED, "batched qr panel: too many rows");
  if ((int64_t)njobs * cs > 0x7fffffff) return fail(TT_ERR_UNSUPPORTED, "batched qr panel: too many jobs");
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(njobs * cs));
  cfg.blockDim = dim3(PT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = cs > 1 ? 1 : 0;
  auto go = [&](auto kernel) -> int {
    TT_TRY(allow_smem(kernel, kPanelSmemMax));
    TT_CUDA_CHECK(cudaLaunchKernelEx(&cfg, kernel, d_jobs, j0, nb));
    note_launch();
    return TT_OK;
  };
  if (nb == 16) {
    if (cs == 1) return go(panel_fast_batched_kernel<TIO, 16, 1>);
    if (cs == 2) return go(panel_fast_batched_kernel<TIO, 16, 2>);
    if (cs == 4) return go(panel_fast_batched_kernel<TIO, 16, 4>);
    return go(panel_fast_batched_kernel<TIO, 16, 8>);
  }
  if (nb == 32) {
    if (cs == 1) return go(panel_fast_batched_kernel<TIO, 32, 1>);
    if (cs == 2) return go(panel_fast_batched_kernel<TIO, 32, 2>);
    if (cs == 4) return go(panel_fast_batched_kernel<TIO, 32, 4>);
    return go(panel_fast_batched_kernel<TIO, 32, 8>);
  }
  return fail(TT_ERR_UNSUPPORTED, "batched qr panel: width must be 16 or 32");
}

template int qr_panel_fast<double>(cudaStream_t, double*, int, int, int, int, int, double*, double*, int, double*,
                                   int);
template int qr_panel_fast<float>(cudaStream_t, float*, int, int, int, int, int, float*, double*, int, float*, int);
template int apply_block_reflector<double>(cudaStream_t, const double*, int, int, int, const double*, int, bool,
                                           double*, int, int);
template int apply_block_reflector<float>(cudaStream_t, const float*, int, int, int, const double*, int, bool,
                                          float*, int, int);
template int qr_panel_fast_batched<double>(cudaStream_t, int, const PanelJob*, int, int, int);
template int qr_panel_fast_batched<float>(cudaStream_t, int, const PanelJob*, int, int, int);

}  // namespace tt
