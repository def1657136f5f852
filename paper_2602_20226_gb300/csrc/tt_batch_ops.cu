// Batched elementwise maps of the batched rounding driver: one job per train, every
// job a strided 2D map dst(i, j) = op(src(i, j)) with its own shape and strides.
// Covers the copies, transposes, R extractions and precision conversions of the sweep.
#include "tt_kernels.cuh"

namespace tt {

namespace {

template <typename TS, typename TD>
__global__ void __launch_bounds__(256) map_batched_kernel(const MapJob* __restrict__ jobs) {
  const MapJob J = jobs[blockIdx.y];
  const int64_t total = (int64_t)J.rows * J.cols;
  if (total <= 0) return;
  const TS* src = static_cast<const TS*>(J.src);
  TD* dst = static_cast<TD*>(J.dst);
  const bool i_fast = (J.dr == 1);  // keep the writes coalesced
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int i, j;
    if (i_fast) {
      i = (int)(e % J.rows);
      j = (int)(e / J.rows);
    } else {
      j = (int)(e % J.cols);
      i = (int)(e / J.cols);
    }
    double v;
    if (J.op == MAP_NS) {
      v = (i == j ? 1.5 : 0.0) - 0.5 * (double)src[i * J.sr + j * J.sc];
    } else if (J.op == MAP_UPPER && i > j) {
      v = 0.0;
    } else {
      v = (double)src[i * J.sr + j * J.sc];
    }
    dst[i * J.dr + j * J.dc] = (TD)v;
  }
}

template <typename T>
__global__ void __launch_bounds__(1024) norm_batched_kernel(const NormJob* __restrict__ jobs) {
  __shared__ double scratch[32];
  const NormJob J = jobs[blockIdx.x];
  const T* a = static_cast<const T*>(J.src);
  double s = 0.0;
  for (int64_t e = threadIdx.x; e < J.n; e += blockDim.x) {
    const double v = (double)a[e];
    s = fma(v, v, s);
  }
  s = block_sum(s, scratch);
  if (threadIdx.x == 0) *J.out = sqrt(s);
}

}  // namespace

template <typename TS, typename TD>
int map_batched(cudaStream_t s, int nj, const MapJob* d_jobs, int64_t max_elems) {
  if (nj <= 0 || max_elems <= 0) return TT_OK;
  if (nj > 65535) return fail(TT_ERR_UNSUPPORTED, "map_batched: too many jobs");
  const unsigned bx = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(max_elems, 256), 512));
  map_batched_kernel<TS, TD><<<dim3(bx, (unsigned)nj), 256, 0, s>>>(d_jobs);
  TT_LAUNCH_CHECK();
  return TT_OK;
}

template <typename T>
int norm_batched(cudaStream_t s, int nj, const NormJob* d_jobs) {
  if (nj <= 0) return TT_OK;
  norm_batched_kernel<T><<<nj, 1024, 0, s>>>(d_jobs);
  TT_LAUNCH_CHECK();
  return TT_OK;
}

template int map_batched<double, double>(cudaStream_t, int, const MapJob*, int64_t);
template int map_batched<float, float>(cudaStream_t, int, const MapJob*, int64_t);
template int map_batched<float, double>(cudaStream_t, int, const MapJob*, int64_t);
template int map_batched<double, float>(cudaStream_t, int, const MapJob*, int64_t);
template int norm_batched<double>(cudaStream_t, int, const NormJob*);
template int norm_batched<float>(cudaStream_t, int, const NormJob*);

}  // namespace tt
