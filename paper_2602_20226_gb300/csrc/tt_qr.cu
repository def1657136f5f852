// Blocked Householder QR of a column-major m x n matrix (used by both rounding sweeps).
//
// Per panel of nb columns: the FP64 panel kernel (tt_panel.cu; one cluster barrier per
// column, FP32 matrices factored in FP64 and rounded back with T recomputed from the rounded
// reflectors), then the trailing update A <- (I - V T^T V^T) A.  The thin Q is formed as
// Q = H_1 ... H_p [I; 0] by the same block-reflector application, panels in reverse.
//
// One train (householder_qr / form_thin_q): the update is one launch per panel
// (apply_block_reflector).  A batch of trains (householder_qr_batched /
// form_thin_q_batched): the panels of all jobs in one launch, the updates as dense batched
// GEMMs over all jobs - FP64: W2 = T^T V^T X by one CTA per column, X -= V W2; FP32 (the
// mixed form): W1 = V^T X by compensated FP32 dot products into FP64, W2 = op(T) W1 in FP64,
// X -= V W2 with W2 split into two FP32 words (exact products, float-float sums).
#include <cooperative_groups.h>

#include <type_traits>

#include "tt_kernels.cuh"
#include "tt_qr.cuh"
#include "tt_panel.cuh"

namespace cg = cooperative_groups;

namespace tt {

namespace {

// W2[:, c] = op(T) (V^T A[:, c]) for one column c per CTA, jb <= 32:
// the small-M half of applying the block reflector I - V T V^T (op(T) = T^T when
// building R, T when building Q).  V (mr x jb) and A (mr x nc) are column-major.
template <typename T, int NT>
__device__ __forceinline__ void reflector_w_body(const T* __restrict__ V, int ldv, const T* __restrict__ A,
                                                 int lda, int mr, int jb, const T* __restrict__ Tm, int ldt,
                                                 bool transpose_t, T* __restrict__ W2, int c) {
  constexpr int NW = NT / 32;
  __shared__ T red[NW][33];
  __shared__ T w[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const T* a = A + (int64_t)c * lda;
  T acc[32];
#pragma unroll
  for (int t = 0; t < 32; ++t) acc[t] = T(0);
  for (int i = tid; i < mr; i += NT) {
    const T ai = a[i];
#pragma unroll
    for (int t = 0; t < 32; ++t)
      if (t < jb) acc[t] += V[i + (int64_t)t * ldv] * ai;
  }
  warp_reduce_scatter32(acc, lane);
  red[warp][lane] = acc[0];
  __syncthreads();
  if (tid < 32) {
    T v = T(0);
#pragma unroll
    for (int q = 0; q < NW; ++q) v += red[q][tid];
    w[tid] = v;
  }
  __syncthreads();
  if (tid < jb) {
    T v = T(0);
    if (transpose_t) {  // (T^T w)_t = sum_{q <= t} T[q, t] w_q
      for (int q = 0; q <= tid; ++q) v += Tm[q + (int64_t)tid * ldt] * w[q];
    } else {  // (T w)_t = sum_{q >= t} T[t, q] w_q
      for (int q = tid; q < jb; ++q) v += Tm[tid + (int64_t)q * ldt] * w[q];
    }
    W2[tid + (int64_t)c * jb] = v;
  }
}

// Batched W2 of the panel at j0 (blockIdx.y = job, blockIdx.x = column): the trailing
// update of the QR (formq = false) or the update of the thin Q being formed.
template <typename T, int NT>
__global__ void __launch_bounds__(NT) reflector_w_batched_kernel(const QrJob<T>* __restrict__ jobs, int j0,
                                                                 int nb, bool formq) {
  const QrJob<T> J = jobs[blockIdx.y];
  const int p = min(J.m, J.n);
  if (j0 >= p) return;
  const int jb = min(nb, p - j0), mr = J.m - j0, c = blockIdx.x;
  const T* V = J.vbuf + j0 + (int64_t)j0 * J.ldv;
  const T* Tm = J.tmat + (int64_t)(j0 / nb) * nb * nb;
  if (!formq) {
    if (c >= J.n - (j0 + jb)) return;
    reflector_w_body<T, NT>(V, J.ldv, J.A + j0 + (int64_t)(j0 + jb) * J.lda, J.lda, mr, jb, Tm, nb, true, J.w2, c);
  } else {
    if (c >= p - j0) return;
    reflector_w_body<T, NT>(V, J.ldv, J.Q + j0 + (int64_t)j0 * J.ldq, J.ldq, mr, jb, Tm, nb, false, J.w2, c);
  }
}

template <typename T>
__global__ void init_thin_q_batched_kernel(const QrJob<T>* __restrict__ jobs) {
  const QrJob<T> J = jobs[blockIdx.y];
  const int p = min(J.m, J.n);
  const int64_t total = (int64_t)J.m * p;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % J.m), c = (int)(e / J.m);
    J.Q[i + (int64_t)c * J.ldq] = (i == c) ? T(1) : T(0);
  }
}

template <typename T>
__global__ void init_thin_q_kernel(T* Q, int m, int p, int ldq) {
  const int64_t total = (int64_t)m * p;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % m), c = (int)(e / m);
    Q[i + (int64_t)c * ldq] = (i == c) ? T(1) : T(0);
  }
}

}  // namespace

// T factors of the panels in FP64: the FP64 form's own, the mixed form's recomputed copy
template <typename T>
double* tmat_f64(const QrWork<T>& w) {
  if constexpr (std::is_same<T, double>::value) return w.tmat;
  else return w.tmat64;
}

template <typename T>
int householder_qr(cudaStream_t s, T* A, int m, int n, int lda, QrWork<T>& w) {
  const int p = std::min(m, n);
  const int nb = w.nb;
  double* tm = tmat_f64(w);
  if (!tm) return fail(TT_ERR_WORKSPACE, "householder_qr: no FP64 T buffer");
  int panel = 0;
  for (int j0 = 0; j0 < p; j0 += nb, ++panel) {
    const int jb = std::min(nb, p - j0);
    double* Tm = tm + (int64_t)panel * nb * nb;
    const int mr = m - j0;
    TT_TRY(qr_panel_fast<T>(s, A, lda, m, j0, jb, nb, w.tau, Tm, nb, w.vbuf, w.ldv));
    const int nt = n - (j0 + jb);
    if (nt <= 0) continue;
    // A_t <- (I - V T^T V^T) A_t
    TT_TRY(apply_block_reflector<T>(s, w.vbuf + j0 + (int64_t)j0 * w.ldv, w.ldv, mr, jb, Tm, nb, true,
                                    A + j0 + (int64_t)(j0 + jb) * lda, lda, nt));
  }
  w.m = m;
  w.n = n;
  w.npanels = panel;
  return TT_OK;
}

template <typename T>
int form_thin_q(cudaStream_t s, const QrWork<T>& w, T* Q, int ldq) {
  const int m = w.m, p = std::min(w.m, w.n), nb = w.nb;
  {
    const int64_t total = (int64_t)m * p;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(total, 256), 8192));
    init_thin_q_kernel<T><<<blocks, 256, 0, s>>>(Q, m, p, ldq);
    TT_LAUNCH_CHECK();
  }
  const double* tm = tmat_f64(w);
  for (int panel = w.npanels - 1; panel >= 0; --panel) {
    const int j0 = panel * nb;
    const int jb = std::min(nb, p - j0);
    // Q_s <- (I - V T V^T) Q_s
    TT_TRY(apply_block_reflector<T>(s, w.vbuf + j0 + (int64_t)j0 * w.ldv, w.ldv, m - j0, jb,
                                    tm + (int64_t)panel * nb * nb, nb, false, Q + j0 + (int64_t)j0 * ldq, ldq,
                                    p - j0));
  }
  return TT_OK;
}

// ---------------------------------------------------------------- batched QR
// The GEMMs that apply the panel at j0 of every job to its trailing block X (mr x nc,
// column-major, ld ldx): W1 = V^T X, W2 = op(T) W1, X -= V W2, as dense batched launches
// over all jobs (a CTA per column would re-read the whole mr x jb reflector panel, tens of
// GB of L2 traffic per panel for hundreds of jobs; a tile reads it once).  FP64 jobs form
// W2 by the reflector kernel (one CTA per column: there the FP64 pipe, not L2, is the
// limit) and run only the update as a GEMM.  FP32 jobs run all three: W1 by Dot2 into
// FP64, W2 in FP64 with the FP64 T factor of the panel, and the update with W2 split into
// two FP32 words - the rounding of W1, W2 or T to FP32 each left the mixed form above
// 1e-6 on the longer trains of the uneven batch.
template <typename T>
struct UpdTypes;
template <>
struct UpdTypes<double> {
  using J1 = GemmJob<double, double, double>;
  using J2 = GemmJob<double, double, double>;
  using J3 = GemmJob<double, double, double>;
};
template <>
struct UpdTypes<float> {
  using J1 = GemmJob<float, float, double>;
  using J2 = GemmJob<double, double, double>;
  using J3 = GemmJob<float, double, float>;
};

template <typename T>
struct PanelGemms {
  std::vector<typename UpdTypes<T>::J1> w1;
  std::vector<typename UpdTypes<T>::J2> w2;
  std::vector<typename UpdTypes<T>::J3> up;
  int n1 = 0;
  TilePlan p1, p2, p3;  // dense tile plans of the three GEMMs
};

template <typename T>
double* tmat_f64(const QrJob<T>& J) {
  if constexpr (std::is_same<T, double>::value) return J.tmat;
  else return J.tmat64;
}

template <typename T>
void panel_gemm_jobs(const QrJob<T>& J, int j0, int nb, bool formq, PanelGemms<T>& G) {
  using J1 = typename UpdTypes<T>::J1;
  using J2 = typename UpdTypes<T>::J2;
  using J3 = typename UpdTypes<T>::J3;
  const int p = std::min(J.m, J.n);
  T* X = nullptr;
  int ldx = 0, nc = 0;
  const int jb = j0 < p ? std::min(nb, p - j0) : 0, mr = J.m - j0;
  if (j0 < p) {
    if (!formq) {
      X = J.A + j0 + (int64_t)(j0 + jb) * J.lda;
      ldx = J.lda;
      nc = J.n - (j0 + jb);
    } else {
      X = J.Q + j0 + (int64_t)j0 * J.ldq;
      ldx = J.ldq;
      nc = p - j0;
    }
  }
  if (nc <= 0) {
    G.w1.push_back(J1{});
    G.w2.push_back(J2{});
    G.up.push_back(J3{});
    return;
  }
  const T* V = J.vbuf + j0 + (int64_t)j0 * J.ldv;
  if constexpr (std::is_same<T, double>::value) {
    G.w1.push_back(J1{});
    G.w2.push_back(J2{});
    G.up.push_back(J3{V, J.w2, X, 1, J.ldv, 1, jb, 1, ldx, mr, nc, jb, -1.0, 1.0});
  } else {
    const double* Tm = J.tmat64 + (int64_t)(j0 / nb) * nb * nb;
    // W1 (jb x nc, ld jb) = V^T X
    G.w1.push_back(J1{V, X, J.w1d, J.ldv, 1, 1, ldx, 1, jb, jb, nc, mr, 1.0, 0.0});
    // W2 = T^T W1 (QR of A) or T W1 (building Q); T is upper triangular, zero below
    if (!formq) G.w2.push_back(J2{Tm, J.w1d, J.w2d, nb, 1, 1, jb, 1, jb, jb, nc, jb, 1.0, 0.0});
    else G.w2.push_back(J2{Tm, J.w1d, J.w2d, 1, nb, 1, jb, 1, jb, jb, nc, jb, 1.0, 0.0});
    // X -= V W2
    G.up.push_back(J3{V, J.w2d, X, 1, J.ldv, 1, jb, 1, ldx, mr, nc, jb, -1.0, 1.0});
  }
  G.n1 = std::max(G.n1, nc);
}

template <typename T>
struct PanelArrays {
  const typename UpdTypes<T>::J1* d1 = nullptr;
  const typename UpdTypes<T>::J2* d2 = nullptr;
  const typename UpdTypes<T>::J3* d3 = nullptr;
  const int *e1 = nullptr, *e2 = nullptr, *e3 = nullptr;
};

// d1..d3: the GEMM jobs of every panel ([panel][job]); e1..e3: their tile prefixes
// ([panel][job + 1]).
template <typename T>
int apply_panels(cudaStream_t s, const QrJob<T>* d_jobs, int nj, int nb, bool formq, int pn, const PanelArrays<T>& D,
                 const std::vector<PanelGemms<T>>& meta, unsigned* status) {
  const PanelGemms<T>& M = meta[pn];
  if (M.n1 <= 0) return TT_OK;
  const size_t jo = (size_t)pn * nj, po = (size_t)pn * (nj + 1);
  if constexpr (std::is_same<T, float>::value) {
    TT_TRY(gemm_batched_dense(s, nj, D.d1 + jo, D.e1 + po, M.p1, true, status));
    TT_TRY(gemm_batched_dense(s, nj, D.d2 + jo, D.e2 + po, M.p2, true, status));
  } else {
    reflector_w_batched_kernel<T, 256><<<dim3((unsigned)M.n1, (unsigned)nj), 256, 0, s>>>(d_jobs, pn * nb, nb,
                                                                                          formq);
    TT_LAUNCH_CHECK();
  }
  return gemm_batched_dense(s, nj, D.d3 + jo, D.e3 + po, M.p3, true, status);
}

template <typename T>
int build_panel_gemms(cudaStream_t s, const std::vector<QrJob<T>>& hj, int nb, bool formq, int npanels,
                      JobArena& arena, std::vector<PanelGemms<T>>& meta, PanelArrays<T>& D) {
  const int nj = (int)hj.size();
  meta.assign(npanels, PanelGemms<T>{});
  std::vector<typename UpdTypes<T>::J1> a1;
  std::vector<typename UpdTypes<T>::J2> a2;
  std::vector<typename UpdTypes<T>::J3> a3;
  std::vector<int> q1((size_t)npanels * (nj + 1)), q2(q1.size()), q3(q1.size());
  for (int pn = 0; pn < npanels; ++pn) {
    PanelGemms<T>& M = meta[pn];
    for (const auto& J : hj) panel_gemm_jobs(J, pn * nb, nb, formq, M);
    const size_t po = (size_t)pn * (nj + 1);
    M.p1 = tile_prefix(M.w1.data(), nj, q1.data() + po);
    M.p2 = tile_prefix(M.w2.data(), nj, q2.data() + po);
    M.p3 = tile_prefix(M.up.data(), nj, q3.data() + po);
    a1.insert(a1.end(), M.w1.begin(), M.w1.end());
    a2.insert(a2.end(), M.w2.begin(), M.w2.end());
    a3.insert(a3.end(), M.up.begin(), M.up.end());
  }
  D.d1 = arena.push(a1, s);
  D.d2 = arena.push(a2, s);
  D.d3 = arena.push(a3, s);
  D.e1 = arena.push(q1, s);
  D.e2 = arena.push(q2, s);
  D.e3 = arena.push(q3, s);
  if (!D.d1 || !D.d2 || !D.d3 || !D.e1 || !D.e2 || !D.e3) return fail(TT_ERR_WORKSPACE, "batched QR: job arena full");
  return TT_OK;
}

template <typename T>
int householder_qr_batched(cudaStream_t s, const std::vector<QrJob<T>>& hj, const QrJob<T>* d_jobs, int nb,
                           JobArena& arena, unsigned* status) {
  const int nj = (int)hj.size();
  if (nj == 0) return TT_OK;
  if (nj > 65535) return fail(TT_ERR_UNSUPPORTED, "householder_qr_batched: too many jobs");
  int p_max = 0;
  std::vector<PanelJob> pj;
  for (const auto& J : hj) {
    p_max = std::max(p_max, std::min(J.m, J.n));
    pj.push_back(PanelJob{J.A, J.m, J.n, J.lda, J.tau, tmat_f64(J), J.vbuf, J.ldv});
  }
  const PanelJob* d_pj = arena.push(pj, s);
  if (!d_pj) return fail(TT_ERR_WORKSPACE, "batched QR: job arena full");
  const int npanels = (int)ceil_div(p_max, nb);
  std::vector<PanelGemms<T>> meta;
  PanelArrays<T> D;
  TT_TRY(build_panel_gemms(s, hj, nb, false, npanels, arena, meta, D));
  for (int pn = 0; pn < npanels; ++pn) {
    const int j0 = pn * nb;
    int mr_max = 0;
    for (const auto& J : hj)
      if (j0 < std::min(J.m, J.n)) mr_max = std::max(mr_max, J.m - j0);
    TT_TRY(qr_panel_fast_batched<T>(s, nj, d_pj, j0, nb, mr_max));
    TT_TRY(apply_panels(s, d_jobs, nj, nb, false, pn, D, meta, status));
  }
  return TT_OK;
}

template <typename T>
int form_thin_q_batched(cudaStream_t s, const std::vector<QrJob<T>>& hj, const QrJob<T>* d_jobs, int nb,
                        JobArena& arena, unsigned* status) {
  const int nj = (int)hj.size();
  if (nj == 0) return TT_OK;
  int p_max = 0;
  int64_t qmax = 1;
  for (const auto& J : hj) {
    const int p = std::min(J.m, J.n);
    p_max = std::max(p_max, p);
    qmax = std::max<int64_t>(qmax, (int64_t)J.m * p);
  }
  init_thin_q_batched_kernel<T><<<dim3((unsigned)std::min<int64_t>(ceil_div(qmax, 256), 1024), (unsigned)nj), 256,
                                  0, s>>>(d_jobs);
  TT_LAUNCH_CHECK();
  const int npanels = (int)ceil_div(p_max, nb);
  std::vector<PanelGemms<T>> meta;
  PanelArrays<T> D;
  TT_TRY(build_panel_gemms(s, hj, nb, true, npanels, arena, meta, D));
  for (int pn = npanels - 1; pn >= 0; --pn) TT_TRY(apply_panels(s, d_jobs, nj, nb, true, pn, D, meta, status));
  return TT_OK;
}

template int householder_qr_batched<double>(cudaStream_t, const std::vector<QrJob<double>>&, const QrJob<double>*,
                                            int, JobArena&, unsigned*);
template int householder_qr_batched<float>(cudaStream_t, const std::vector<QrJob<float>>&, const QrJob<float>*,
                                           int, JobArena&, unsigned*);
template int form_thin_q_batched<double>(cudaStream_t, const std::vector<QrJob<double>>&, const QrJob<double>*,
                                         int, JobArena&, unsigned*);
template int form_thin_q_batched<float>(cudaStream_t, const std::vector<QrJob<float>>&, const QrJob<float>*,
                                        int, JobArena&, unsigned*);
template int householder_qr<double>(cudaStream_t, double*, int, int, int, QrWork<double>&);
template int householder_qr<float>(cudaStream_t, float*, int, int, int, QrWork<float>&);
template int form_thin_q<double>(cudaStream_t, const QrWork<double>&, double*, int);
template int form_thin_q<float>(cudaStream_t, const QrWork<float>&, float*, int);

}  // namespace tt
