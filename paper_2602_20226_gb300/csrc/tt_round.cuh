// TT rounding driver.
#pragma once

#include <algorithm>
#include <cmath>
#include <type_traits>

#include "tt_common.cuh"
#include "tt_qr.cuh"
#include "tt_svd.cuh"

namespace tt {

// ---- scratch layout of one rounding (shared by tt_round and the batched driver)
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
  int64_t d_max = 1;  // largest mode
};

inline Dims dims_of(const tt_train* x) {
  Dims D;
  D.L = x->L;
  for (int k = 0; k < x->L; ++k) {
    D.S_max = std::max<int64_t>(D.S_max, x->ranks[k] * (int64_t)x->d[k] * x->ranks[k + 1]);
    D.r_max = std::max<int64_t>(D.r_max, std::max(x->ranks[k], x->ranks[k + 1]));
    D.d_max = std::max<int64_t>(D.d_max, x->d[k]);
  }
  return D;
}

template <typename T>
struct Bufs {
  T *A = nullptr, *Q = nullptr, *tmp = nullptr, *Rbuf = nullptr, *vsel = nullptr, *F = nullptr;
  float *X32 = nullptr, *G32 = nullptr;  // mixed-form bond SVD: FP32 factor, Newton-Schulz Gram
  // mixed form: FP64 scratch of the preconditioning QR of the square factor
  double* tmp64 = nullptr;
  QrWork<double> qr64;
  // mixed form: W1 = V^T X and W2 = op(T) W1 of the batched driver's QR updates, in FP64
  double *w1d = nullptr, *w2d = nullptr;
  QrWork<T> qr;
  SvdWork sv;
};

// batched: the scratch of a train of tt_apply_round_batched (the FP64 W buffers of the
// mixed form's batched QR updates; tt_round's own updates need none)
template <typename T>
size_t carve(Carver& c, const Dims& D, int nb, Bufs<T>& B, bool batched = false) {
  B.A = c.take<T>(D.S_max);
  B.Q = c.take<T>(D.S_max);
  B.tmp = c.take<T>(D.S_max);
  B.qr.nb = nb;
  B.qr.vbuf = c.take<T>(D.S_max);
  B.qr.tau = c.take<T>(D.r_max + 32);
  B.qr.tmat = c.take<T>((size_t)nb * nb * (ceil_div(D.r_max, nb) + 1));
  if (std::is_same<T, float>::value) B.qr.tmat64 = c.take<double>((size_t)nb * nb * (ceil_div(D.r_max, nb) + 1));
  B.qr.w1 = c.take<T>((size_t)nb * D.r_max);
  B.qr.w2 = c.take<T>((size_t)nb * D.r_max);
  B.Rbuf = c.take<T>((size_t)D.r_max * D.r_max);
  B.vsel = c.take<T>((size_t)D.r_max * D.r_max);
  B.F = c.take<T>((size_t)D.r_max * D.r_max);
  B.sv.X = c.take<double>((size_t)D.r_max * D.r_max);
  if (std::is_same<T, float>::value) {
    B.X32 = c.take<float>((size_t)D.r_max * D.r_max);
    B.G32 = c.take<float>((size_t)D.r_max * D.r_max);
    if (!batched) {
      B.tmp64 = c.take<double>((size_t)D.r_max * D.r_max);
      B.qr64.nb = 16;
      B.qr64.vbuf = c.take<double>((size_t)D.r_max * D.r_max);
      B.qr64.tau = c.take<double>(D.r_max + 32);
      B.qr64.tmat = c.take<double>((size_t)16 * 16 * (ceil_div(D.r_max, 16) + 1));
    }
    if (batched) {
      B.w1d = c.take<double>((size_t)nb * D.r_max);
      B.w2d = c.take<double>((size_t)nb * D.r_max);
    }
  }
  B.sv.sigma = c.take<double>(D.r_max);
  B.sv.perm = c.take<int>(D.r_max);
  B.sv.rank = c.take<int>(2);
  B.sv.sweeps = B.sv.rank + 1;  // next to the rank: one read-back per bond
  B.sv.bar = c.take<unsigned>(2);
  B.sv.rot = c.take<unsigned>(SvdWork::kMaxSweeps);
  B.sv.status = c.take<unsigned>(1);
  B.qr.status = B.sv.status;
  B.sv.norm = c.take<double>(1);
  B.sv.epoch = c.take<unsigned>((size_t)D.r_max + 2);
  return c.off + 256;
}

// Householder panel width: 16 columns, except the batched driver's mixed form (32: its QR
// updates run as dense batched GEMMs over all jobs, and the wider panels carry its largest
// trains' error further below 1e-6); the single-train mixed form takes 16, whose panels cost
// about half per column (emulated error on the 2D rank-64 train 5.0e-7 -> 5.5e-7)
template <typename T>
inline int panel_width(bool batched = false) {
  return sizeof(T) == 8 ? 16 : (batched ? 32 : 16);
}

// Relative resolution of the mixed form's bond SVD (see the truncation call).
constexpr double kMixedSigmaFloor = 1.0 / (1 << 22);

template <typename T>
inline double jacobi_tol(int nrow) {
  // columns are treated as orthogonal once |x_a . x_b| <= tol ||x_a|| ||x_b||
  return std::sqrt((double)std::max(nrow, 1)) * 2.220446049250313e-16;
}


struct RoundStats {
  int jacobi_sweeps = 0;
};

// Intermediates of one FP64 rounding, recorded for its adjoint (tt_round_backward): device
// copies in a caller-given arena, host sizes alongside.  All matrices FP64; "cm" = column-major.
struct RoundRecord {
  char* base = nullptr;
  size_t cap = 0, off = 0;
  bool overflow = false;
  struct RL {     // right-to-left step at site k: dt = D_k^T (m x n cm) = q r
    int m = 0, n = 0, p = 0, rows_prev = 0;
    double *dt = nullptr, *q = nullptr, *r = nullptr;  // q: m x p cm, r: p x n cm
    double* xprev = nullptr;                           // core k-1 before the step (rows_prev x n)
  };
  struct LR {     // left-to-right bond k: a = C_k (m x n row-major) before the bond
    int m = 0, n = 0, p = 0, rn = 0, cols_next = 0;
    bool tall = true, cert = false;
    double *a = nullptr, *q = nullptr, *r = nullptr;     // tall: q (m x p cm), r (p x n cm)
    double *u = nullptr, *sigma = nullptr, *f = nullptr;  // SVD bonds: U of the square factor
                                                          // (p x p cm, sorted), sigma (p), F (rn x n)
    double* next = nullptr;                               // C_{k+1} before the bond (n x cols_next)
  };
  std::vector<RL> rl;
  std::vector<LR> lr;
  double* take(size_t n) {
    off = (off + 255) & ~size_t(255);
    if (off + n * sizeof(double) > cap) {
      overflow = true;
      return nullptr;
    }
    double* p = reinterpret_cast<double*>(base + off);
    off += n * sizeof(double);
    return p;
  }
};
// arena bytes that recording the rounding of x needs (an upper bound)
size_t round_record_bytes(const tt_train* x);

size_t round_workspace_bytes(const tt_train* x, int prec, bool batched = false);

template <typename T>
int round_impl(const tt_train* x, double eps, int64_t max_rank, tt_train* out, double* norm_out,
               void* ws, size_t ws_bytes, cudaStream_t s, RoundStats* stats, RoundRecord* rec = nullptr);

// adjoint of the FP64 rounding (tt_round_bwd.cu)
size_t round_backward_workspace_bytes(const tt_train* x);
int round_backward_impl(const tt_train* x, double eps, int64_t max_rank, const tt_train* dout, tt_train* dx,
                        void* ws, size_t ws_bytes, cudaStream_t s);

size_t batched_workspace_bytes(int32_t n, const tt_mpo* W, const tt_train* x, int32_t prec);
int apply_round_batched(int32_t n, const tt_mpo* W, const tt_train* x, tt_train* y, double eps,
                        int64_t max_rank, int32_t prec, tt_train* out, void* ws, size_t ws_bytes,
                        void* const* streams, int32_t nstreams);

}  // namespace tt
