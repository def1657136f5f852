// Shared device/host helpers of libtt (sm_103a).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstring>
#include <vector>
#include <stdint.h>

#include <string>

#include "../../include/tt.h"

namespace tt {

// ---------------------------------------------------------------- host errors

void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
void note_launch();  // counts kernel launches made by the library (tt_launch_count)

// opt-in event profiler of tt_round's phases (tt_profile_enable / tt_profile_read)
enum ProfClass { PROF_JACOBI = 0, PROF_QR = 1, PROF_GEMM = 2, PROF_CERT = 3, PROF_CLASSES = 4 };
bool profile_enabled();
void profile_add(int cls, double ms, double flops, double executed);

#define TT_CUDA_CHECK(expr)                                                             \
  do {                                                                                  \
    cudaError_t _e = (expr);                                                            \
    if (_e != cudaSuccess)                                                              \
      return ::tt::fail(TT_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
  } while (0)

// after a <<<...>>> launch: count it and check the launch error
#define TT_LAUNCH_CHECK()                    \
  do {                                       \
    ::tt::note_launch();                     \
    TT_CUDA_CHECK(cudaGetLastError());       \
  } while (0)

#define TT_TRY(...)                 \
  do {                              \
    int _s = (__VA_ARGS__);         \
    if (_s != TT_OK) return _s;     \
  } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

int num_sms();

// ----------------------------------------------------------- device status word
// Bit flags a kernel may raise; the host reads them at the next synchronisation.
enum : unsigned {
  ST_NONCONVERGED = 1u,  // Jacobi sweep cap reached
  ST_TIMEOUT = 2u,       // bounded wait expired
  ST_NONFINITE = 4u,     // NaN / Inf met
  ST_BAD_INDEX = 8u      // an index argument was out of range (access skipped)
};

// ---------------------------------------------------------- warp reductions

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// ---------------------------------------------------- thread-block cluster helpers
// Cluster-wide barrier with release/acquire semantics, as explicit PTX with a memory
// clobber so that no shared-memory access moves across it.
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

// Load of `*p` from the shared memory of CTA `rank` of this cluster (distributed shared
// memory).  Spelled out as mapa + ld.shared::cluster: a plain dereference of a mapped
// generic pointer let the compiler schedule the load ahead of the preceding cluster
// barrier, so CTAs read partials that their peers had not written yet.
__device__ __forceinline__ double dsmem_load(const double* p, int rank) {
  unsigned a = (unsigned)__cvta_generic_to_shared(p), ra;
  double v;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(ra) : "memory");
  return v;
}
__device__ __forceinline__ float dsmem_load(const float* p, int rank) {
  unsigned a = (unsigned)__cvta_generic_to_shared(p), ra;
  float v;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(ra) : "memory");
  return v;
}

// Reduce-scatter of 32 values across a warp: on entry lane l holds partials v[0..31];
// on exit v[0] of lane l holds the warp total of index l.  31 shuffles in all.
template <typename T>
__device__ __forceinline__ void warp_reduce_scatter32(T (&v)[32], int lane) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    const bool upper = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < off; ++i) {
      T send = upper ? v[i] : v[i + off];
      T keep = upper ? v[i + off] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
}

// Block-wide sum; every thread gets the total.  `scratch` holds >= 32 values.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  T t = (lane < nwarps) ? scratch[lane] : T(0);
  t = warp_sum(t);
  return t;
}

// --------------------------------------------------------------- bounded waits
// Acquire load of a device word written by another CTA.
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Polls until *word >= target.  After `limit` polls it raises ST_TIMEOUT in *status and
// returns false; it also gives up (false) once another thread has raised ST_TIMEOUT.
constexpr long long kWaitPolls = 1ll << 24;
__device__ __forceinline__ bool bounded_wait_ge(const unsigned* word, unsigned target, unsigned* status,
                                                long long limit = kWaitPolls) {
  long long polls = 0;
  while (ld_acquire_u32(word) < target) {
    if (++polls > limit) {
      atomicOr(status, (unsigned)ST_TIMEOUT);
      return false;
    }
    if ((polls & 255) == 0 && (*(volatile unsigned*)status & ST_TIMEOUT)) return false;
  }
  return true;
}

// ------------------------------------------------------- bounded grid barrier
// Sense-reversing barrier for a cooperative launch (all CTAs co-resident).  Every
// wait is bounded: after `limit` polls the CTA raises ST_TIMEOUT in *status and
// returns false; callers then leave the kernel.  bar[0] = arrival count,
// bar[1] = generation.  Both must be zero-initialised before the launch.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned nblocks, unsigned* status,
                                             long long limit = (1ll << 26)) {
  __syncthreads();
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = bar + 1;
    const unsigned gen = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u);
    int ok = 1;
    if (arrived == nblocks - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long polls = 0;
      while (*vgen == gen) {
        if (++polls > limit) {
          atomicOr(status, (unsigned)ST_TIMEOUT);
          ok = 0;
          break;
        }
        if ((polls & 1023) == 0 && (*(volatile unsigned*)status & ST_TIMEOUT)) {
          ok = 0;  // another CTA gave up already
          break;
        }
        __nanosleep(20);
      }
    }
    __threadfence();
    if (*(volatile unsigned*)status & ST_TIMEOUT) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// ------------------------------------------------------------ batched job arrays
// Per-launch job descriptors of the batched driver: staged in a pinned host ring and
// copied asynchronously into a device region carved from the caller's workspace.
// reset() may be called only when the stream has consumed every pushed array (after
// a stream synchronisation).
struct JobArena {
  char* dev = nullptr;
  char* host = nullptr;  // pinned
  size_t cap = 0, off = 0;
  template <typename J>
  const J* push(const std::vector<J>& v, cudaStream_t s) {
    const size_t bytes = v.size() * sizeof(J);
    const size_t o = (off + 255) & ~size_t(255);
    if (o + bytes > cap) return nullptr;
    if (bytes) {
      std::memcpy(host + o, v.data(), bytes);
      if (cudaMemcpyAsync(dev + o, host + o, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return nullptr;
    }
    off = o + bytes;
    return reinterpret_cast<const J*>(dev + o);
  }
  void reset() { off = 0; }
};

// --------------------------------------------------------------- small types

template <typename T>
struct DTypeOf;
template <>
struct DTypeOf<double> {
  static constexpr int value = TT_F64;
};
template <>
struct DTypeOf<float> {
  static constexpr int value = TT_F32;
};

}  // namespace tt
