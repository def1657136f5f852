// Tensor-core GEMM for the mixed form:  C = alpha * A B + beta * C  with FP32 operands,
// computed on the 5th-generation tensor cores (tcgen05, kind::tf32) with a 3-term
// split so the result keeps ~FP32 accuracy:
//     x = x_hi + x_lo,  x_hi = rn_tf32(x),  x_lo = x - x_hi (exact in FP32)
//     A B ~= A_hi B_hi + A_hi B_lo + A_lo B_hi           (the lo*lo term is < 2^-23)
// (split-precision products: Ootomo & Yokota 2022; Henry, Tang, Heinecke 2019).
//
// One CTA (128 threads = 4 warps) owns a 128 x BN output tile.  The accumulator lives
// in tensor memory (BN FP32 columns x 128 lanes).  Per 32-wide K block, all threads
// load the A and B tiles from global memory, split them and store hi and lo parts in
// shared memory in the no-swizzle K-major canonical layout (8-row x 16-byte core
// matrices); then one thread issues 3 x 4 tcgen05.mma (K = 8 each) into a fresh
// tensor-memory buffer and commits them to an mbarrier.  Two shared-memory stages and
// two accumulator buffers let the loads and MMAs of block k+1 overlap the draining of
// block k's partial into FP32 registers.  Every mbarrier wait is bounded: on expiry the
// kernel raises ST_TIMEOUT, waits (bounded) for its MMAs, frees its tensor memory and
// skips the epilogue.
#include <cstdint>

#include "tt_gemm.cuh"

namespace tt {

namespace {

constexpr int TC_BM = 128, TC_BK = 32, TC_THREADS = 128;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// tcgen05 shared-memory matrix descriptor: start address, leading-dimension byte
// offset (between core matrices along K), stride-dimension byte offset (between
// 8-row groups), descriptor version 1 (bit 46), no swizzle, base offset 0.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor: D = F32, A = B = TF32, both K-major, M = 128, N = bn
__host__ __device__ constexpr uint32_t idesc_tf32(int bn) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(bn >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred P1;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
      "selp.b32 %0, 1, 0, P1;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// bounded wait: ~ a second at most
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (long long i = 0; i < (1ll << 22); ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (i > 64) __nanosleep(64);
  }
  return false;
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(tmem_d), "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
  hi = __uint_as_float(u);
  lo = x - hi;
}

// byte offset of element (row, k) of a rows x 32 K-major no-swizzle tile
__device__ __forceinline__ uint32_t tile_off(int row, int k) {
  return (uint32_t)((row >> 3) * 1024 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

struct TcArgs {
  int M, N, K;
  double alpha, beta;
  const float* A;
  int64_t sam, sak;
  const float* B;
  int64_t sbk, sbn;
  float* C;
  int64_t scm, scn;
  unsigned* status;
};

// Load a rows x 32 tile of an operand whose element (row, k) sits at P[row*srow + k*sk],
// split it and store hi / lo in the canonical layout.  Rows beyond nrows and k beyond K
// are zero.
template <int ROWS>
__device__ __forceinline__ void load_split(const float* __restrict__ P, int64_t srow, int64_t sk,
                                           int row0, int nrows, int k0, int K, uint8_t* hi,
                                           uint8_t* lo) {
  const int tid = threadIdx.x;
  constexpr int PER = ROWS * TC_BK / TC_THREADS;
  if (sk == 1 || srow != 1) {  // k fastest across threads
#pragma unroll 4
    for (int u = 0; u < PER; ++u) {
      const int e = tid + u * TC_THREADS;
      const int k = e & 31, r = e >> 5;
      const int gr = row0 + r, gk = k0 + k;
      const float v = (gr < nrows && gk < K) ? __ldg(P + (int64_t)gr * srow + (int64_t)gk * sk) : 0.0f;
      float h, l;
      split_tf32(v, h, l);
      const uint32_t o = tile_off(r, k);
      *reinterpret_cast<float*>(hi + o) = h;
      *reinterpret_cast<float*>(lo + o) = l;
    }
  } else {  // rows fastest across threads
#pragma unroll 4
    for (int u = 0; u < PER; ++u) {
      const int e = tid + u * TC_THREADS;
      const int r = e % ROWS, k = e / ROWS;
      const int gr = row0 + r, gk = k0 + k;
      const float v = (gr < nrows && gk < K) ? __ldg(P + (int64_t)gr * srow + (int64_t)gk * sk) : 0.0f;
      float h, l;
      split_tf32(v, h, l);
      const uint32_t o = tile_off(r, k);
      *reinterpret_cast<float*>(hi + o) = h;
      *reinterpret_cast<float*>(lo + o) = l;
    }
  }
}

// Read a finished per-block partial (BN columns of this thread's row) out of tensor
// memory and add it into the FP32 register accumulator with round-to-nearest.
template <int BN, typename Acc>
__device__ __forceinline__ void drain_partial(uint32_t lane_base, Acc (&acc)[BN]) {
#pragma unroll
  for (int c0 = 0; c0 < BN; c0 += 16) {
    uint32_t r[16];
    tmem_ld16(lane_base + (uint32_t)c0, r);
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[c0 + j] += (Acc)__uint_as_float(r[j]);
  }
}

// Acc = float: block partials summed in FP32 registers (round to nearest).
// Acc = double: block partials summed in FP64 registers, so the error of a long K is
// that of one 32-wide block rather than of the whole FP32 accumulation.
template <int BN, typename Acc>
__global__ void __launch_bounds__(TC_THREADS, 1) gemm_tf32x3_kernel(TcArgs g) {
  extern __shared__ __align__(1024) uint8_t smem[];
  constexpr int A_BYTES = TC_BM * TC_BK * 4, B_BYTES = BN * TC_BK * 4;
  constexpr int STAGE = 2 * A_BYTES + 2 * B_BYTES;
  constexpr uint32_t IDESC = idesc_tf32(BN);
  constexpr uint32_t TMEM_COLS = 2 * BN;  // two accumulator buffers
  __shared__ uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * TC_BM, n0 = blockIdx.x * BN;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(&mbar[0]);
    mbar_init(&mbar[1]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);

  // Each 32-wide K block accumulates into a fresh tensor-memory buffer (stage s uses
  // buffer s, columns s*BN ..); while the MMAs of block kb run, the threads drain the
  // partial of block kb-1 into registers.  Keeping every tensor-core accumulation chain
  // to one K block bounds the bias of its non-round-to-nearest accumulation by the
  // size of one block instead of the whole K; the register sums round to nearest.
  Acc acc[BN];
#pragma unroll
  for (int j = 0; j < BN; ++j) acc[j] = Acc(0);
  uint32_t phase0 = 0, phase1 = 0;
  bool ok = true;
  const int nkb = (g.K + TC_BK - 1) / TC_BK;
  for (int kb = 0; kb < nkb && ok; ++kb) {
    const int s = kb & 1;
    // stage s was last read by block kb-2, whose completion was awaited while draining it
    uint8_t* st = smem + s * STAGE;
    uint8_t* a_hi = st;
    uint8_t* a_lo = st + A_BYTES;
    uint8_t* b_hi = st + 2 * A_BYTES;
    uint8_t* b_lo = st + 2 * A_BYTES + B_BYTES;
    const int k0 = kb * TC_BK;
    load_split<TC_BM>(g.A, g.sam, g.sak, m0, g.M, k0, g.K, a_hi, a_lo);
    load_split<BN>(g.B, g.sbn, g.sbk, n0, g.N, k0, g.K, b_hi, b_lo);
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t dbuf = tmem + (uint32_t)(s * BN);
#pragma unroll
      for (int kk = 0; kk < TC_BK / 8; ++kk) {
        const uint32_t off = kk * 256;  // two core matrices along K per MMA
        const uint64_t dah = smem_desc(smem_u32(a_hi) + off, 128, 1024);
        const uint64_t dal = smem_desc(smem_u32(a_lo) + off, 128, 1024);
        const uint64_t dbh = smem_desc(smem_u32(b_hi) + off, 128, 1024);
        const uint64_t dbl = smem_desc(smem_u32(b_lo) + off, 128, 1024);
        mma_tf32(dbuf, dah, dbh, IDESC, kk > 0 ? 1u : 0u);
        mma_tf32(dbuf, dah, dbl, IDESC, 1u);
        mma_tf32(dbuf, dal, dbh, IDESC, 1u);
      }
      mma_commit(&mbar[s]);
    }
    if (kb > 0) {  // drain block kb-1 from buffer s^1
      const int sp = s ^ 1;
      const bool w = sp == 0 ? mbar_wait(&mbar[0], phase0) : mbar_wait(&mbar[1], phase1);
      if (sp == 0) phase0 ^= 1; else phase1 ^= 1;
      ok = __syncthreads_and(w);
      if (ok) {
        tc_fence_after();
        drain_partial<BN, Acc>(lane_base + (uint32_t)(sp * BN), acc);
        tc_fence_before();
      }
    }
  }
  // drain the last block
  if (ok && nkb > 0) {
    const int sp = (nkb - 1) & 1;
    const bool w = sp == 0 ? mbar_wait(&mbar[0], phase0) : mbar_wait(&mbar[1], phase1);
    ok = __syncthreads_and(w);
    if (ok) {
      tc_fence_after();
      drain_partial<BN, Acc>(lane_base + (uint32_t)(sp * BN), acc);
    }
  } else if (!ok) {
    // a wait expired: give the MMAs in flight a bounded chance to finish before freeing
    // tensor memory (both barriers, whatever their phase)
    mbar_wait(&mbar[0], phase0);
    mbar_wait(&mbar[1], phase1);
  }

  if (ok && nkb > 0) {
    const int row = m0 + warp * 32 + lane;
    if (row < g.M) {
#pragma unroll
      for (int j = 0; j < BN; ++j) {
        const int col = n0 + j;
        if (col < g.N) {
          float* p = g.C + (int64_t)row * g.scm + (int64_t)col * g.scn;
          Acc v = (Acc)g.alpha * acc[j];
          if (g.beta != 0.0) v += (Acc)g.beta * (Acc)(*p);
          *p = (float)v;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS)
                 : "memory");
  }
  if (!ok && tid == 0 && g.status) atomicOr(g.status, (unsigned)ST_TIMEOUT);
}

template <int BN>
constexpr size_t tc_smem_bytes() {
  return 2 * (2 * TC_BM * TC_BK * 4 + 2 * BN * TC_BK * 4);
}

template <int BN, typename Acc>
int launch_tc(cudaStream_t s, const TcArgs& a) {
  static std::atomic<int> configured{-1};
  int dev = 0;
  TT_CUDA_CHECK(cudaGetDevice(&dev));
  if (configured != dev) {
    TT_CUDA_CHECK(cudaFuncSetAttribute(gemm_tf32x3_kernel<BN, Acc>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)tc_smem_bytes<BN>()));
    configured = dev;
  }
  dim3 grid((unsigned)ceil_div(a.N, BN), (unsigned)ceil_div(a.M, TC_BM));
  if (grid.y > 65535u) return fail(TT_ERR_UNSUPPORTED, "gemm_tf32x3: M too large");
  gemm_tf32x3_kernel<BN, Acc><<<grid, TC_THREADS, tc_smem_bytes<BN>(), s>>>(a);
  TT_LAUNCH_CHECK();
  return TT_OK;
}


// ======================================================================================
// Sliced form with exact tensor-core sums (an Ozaki-type splitting: Ozaki, Ogita, Oishi,
// Rump 2012; Ootomo, Ozaki, Yokota 2024 for integer tensor cores).
//
// Per 32-wide K block every row of A and every column of B gets its own power of two
// 2^E above its largest magnitude, and each value is cut into three signed integer
// slices, each rounded to nearest (balanced digits):
//     v = 2^(E-9) (h1 + 2^-9 h2 + 2^-18 h3) + d,  |h1| <= 512, |h2|, |h3| <= 256,
//     |d| <= 2^(E-28).
// The slices are small integers, exact in TF32, and the tensor cores form three level
// sums per block
//     L0 = sum h1a h1b,  L1 = sum (h1a h2b + h2a h1b),  L2 = sum (h1a h3b + h2a h2b + h3a h1b)
// whose partial sums are integers of magnitude <= 32 * 2^18 = 2^23 (L0, L1) and
// <= 32 * 5 * 2^16 < 2^24 (L2): representable in FP32, so the accumulation inside the
// tensor core is exact whatever its rounding.  The dropped cross terms (h2 h3, h3 h2,
// h3 h3) and the slice remainders cost at most ~2^-25 of max|a| max|b| per product;
// balanced digits make them zero-mean, so same-sign data gets no bias.  After each block
// the threads read the three levels out of tensor memory, scale them by 2^(Ea+Eb-18)
// (exact) and add them into a float-float (hi, lo) accumulator per output with an
// error-free TwoSum (Knuth).
//
// One CTA of 256 threads (two warpgroups) owns a 128 x SL_BN tile; warpgroup g drains
// columns [g SL_BN/2, (g+1) SL_BN/2) of the tensor-memory lanes of its warps.  Per block
// kb: the operand values arrive by cp.async in a padded staging buffer (issued one block
// ahead), are sliced into the canonical K-major layout of stage kb & 1, and one thread
// issues the block's 24 MMAs into tensor-memory buffer kb & 1 while the threads drain
// block kb-1 from the other buffer.  Every mbarrier wait is bounded, as above.

constexpr int SL_BK = 32, SL_BN = 64, SL_RAW = SL_BK + 1, SL_THREADS = 256;
constexpr int SL_A_BYTES = TC_BM * SL_BK * 4, SL_B_BYTES = SL_BN * SL_BK * 4;
constexpr int SL_STAGE = 3 * SL_A_BYTES + 3 * SL_B_BYTES;
constexpr int SL_RAW_FLOATS = (TC_BM + SL_BN) * SL_RAW;  // one staging buffer: A rows, then B rows
// NST stages (and tensor-memory buffers): 2 for the pipelined K loop, 1 when K fits one
// block (then two CTAs share an SM: shared memory below half of it, 256 TMEM columns)
template <int NST>
__host__ __device__ constexpr size_t sl_smem() {
  return NST * SL_STAGE + NST * SL_RAW_FLOATS * 4 + NST * (TC_BM + SL_BN) * 4;
}
template <int NST>
__host__ __device__ constexpr uint32_t sl_tmem_cols() {
  return NST == 2 ? 512u : 256u;
}
static_assert(2 * 3 * SL_BN <= (int)sl_tmem_cols<2>() && 3 * SL_BN <= (int)sl_tmem_cols<1>(),
              "tensor memory of the level sums");
static_assert(sl_smem<2>() <= 227 * 1024, "shared memory of the sliced GEMM");
static_assert(2 * (sl_smem<1>() + 2048) <= 228 * 1024, "two one-block CTAs per SM");

__device__ __forceinline__ void cp_async4(float* dst, const float* src, int bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Asynchronous copy of one rows x 32 block of an operand whose element (row, k) is
// P[row*srow + k*sk] into raw (row stride SL_RAW): a warp copies 32 consecutive k of one
// row, or 32 consecutive rows of one k when the rows are contiguous.  Zero-filled beyond
// nrows / K (those copies read nothing and point at P itself).
template <int ROWS>
__device__ __forceinline__ void raw_prefetch(const float* __restrict__ P, int64_t srow, int64_t sk, int row0,
                                             int nrows, int k0, int K, float* raw) {
  constexpr int PER = ROWS * SL_BK / SL_THREADS;
  const int tid = threadIdx.x;
  const bool kfast = (sk == 1 || srow != 1);
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int e = tid + u * SL_THREADS;
    const int r = kfast ? (e >> 5) : (e % ROWS), k = kfast ? (e & 31) : (e / ROWS);
    const int gr = row0 + r, gk = k0 + k;
    const bool in = gr < nrows && gk < K;
    cp_async4(raw + r * SL_RAW + k, in ? P + (int64_t)gr * srow + (int64_t)gk * sk : P, in ? 4 : 0);
  }
}

// byte offset of element (row, k) of a rows x 32 K-major no-swizzle tile (8-row x 16-byte
// core matrices, 128 bytes apart along K, 1024 bytes apart along the rows)
__device__ __forceinline__ uint32_t tile32_off(int row, int k) {
  return (uint32_t)((row >> 3) * 1024 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

// Cut the rows x 32 block in raw into three integer slices stored in the canonical layout
// at s0 / s1 / s2, and each row's output scale 2^(E-9) in pscale.  TPR threads share a
// row: lane = part * (32 / TPR) + row-in-warp, so that the staging reads and the 16-byte
// slice stores of a warp hit distinct banks.  A row whose largest magnitude is below
// 2^-118 (or zero) gets zero slices and scale 0.
template <int ROWS>
__device__ __forceinline__ void slice_rows(const float* raw, uint8_t* s0, uint8_t* s1, uint8_t* s2,
                                           float* pscale) {
  constexpr int TPR = SL_THREADS / ROWS;  // threads per row: 2 (A) or 4 (B)
  constexpr int KPT = SL_BK / TPR;        // 16 or 8
  constexpr int RPW = 32 / TPR;           // rows per warp
  static_assert(TPR * ROWS == SL_THREADS && KPT % 4 == 0, "slice layout");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int row = warp * RPW + lane % RPW, part = lane / RPW;
  float v[KPT];
  float m = 0.0f;
#pragma unroll
  for (int j = 0; j < KPT; ++j) {
    v[j] = raw[row * SL_RAW + part * KPT + j];
    m = fmaxf(m, fabsf(v[j]));
  }
#pragma unroll
  for (int off = RPW; off < 32; off <<= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
  // biased exponent eb of the largest magnitude: m < 2^E with E = eb - 126
  const uint32_t eb = __float_as_uint(m) >> 23;
  const bool live = eb >= 9u;
  const float sin = live ? __uint_as_float((262u - eb) << 23) : 0.0f;  // 2^(9 - E)
  const float sout = live ? __uint_as_float((eb - 8u) << 23) : 0.0f;   // 2^(E - 9)
#pragma unroll
  for (int q = 0; q < KPT / 4; ++q) {
    float4 a, b, c;
    float* pa = &a.x;
    float* pb = &b.x;
    float* pc = &c.x;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const float x = __fmul_rn(v[4 * q + t], sin);  // |x| < 2^9, exact
      const float h1 = rintf(x);
      const float y = __fmul_rn(__fsub_rn(x, h1), 512.0f);  // exact (Sterbenz), |y| <= 256
      const float h2 = rintf(y);
      const float z = __fmul_rn(__fsub_rn(y, h2), 512.0f);
      pa[t] = h1;
      pb[t] = h2;
      pc[t] = rintf(z);
    }
    const uint32_t o = tile32_off(row, part * KPT + 4 * q);
    *reinterpret_cast<float4*>(s0 + o) = a;
    *reinterpret_cast<float4*>(s1 + o) = b;
    *reinterpret_cast<float4*>(s2 + o) = c;
  }
  if (part == 0) pscale[row] = sout;
}

__device__ __forceinline__ void tmem_ld16_issue(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

constexpr int SL_HALF = SL_BN / 2;  // columns drained by one warpgroup

// Add one block's three levels (tensor-memory columns buf + l*SL_BN + c of this warp's
// lanes, c in this warpgroup's half) into the float-float accumulators of this thread's
// row; nvalid = columns of this warpgroup's half inside N.
__device__ __forceinline__ void drain_levels(uint32_t lane_base, float pa, const float* pb, int nvalid,
                                             float (&hi)[SL_HALF], float (&lo)[SL_HALF]) {
#pragma unroll
  for (int c0 = 0; c0 < SL_HALF; c0 += 16) {
    if (c0 < nvalid) {  // uniform across the warpgroup
      uint32_t r0[16], r1[16];
      tmem_ld16_issue(lane_base + (uint32_t)c0, r0);
      tmem_ld16_issue(lane_base + (uint32_t)(SL_BN + c0), r1);
      tmem_wait_ld();
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float sc = __fmul_rn(pa, pb[c0 + j]);  // 2^(Ea+Eb-18), exact
        const float t0 = __fmul_rn(__uint_as_float(r0[j]), sc);
        // TwoSum: hi + t0 = ss + e exactly
        const float h = hi[c0 + j];
        const float ss = __fadd_rn(h, t0);
        const float bb = __fsub_rn(ss, h);
        const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(ss, bb)), __fsub_rn(t0, bb));
        hi[c0 + j] = ss;
        lo[c0 + j] = __fmaf_rn(__uint_as_float(r1[j]), __fmul_rn(sc, 0x1p-9f), __fadd_rn(lo[c0 + j], e));
      }
      tmem_ld16_issue(lane_base + (uint32_t)(2 * SL_BN + c0), r0);
      tmem_wait_ld();
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float sc = __fmul_rn(pa, pb[c0 + j]);
        lo[c0 + j] = __fmaf_rn(__uint_as_float(r0[j]), __fmul_rn(sc, 0x1p-18f), lo[c0 + j]);
      }
    }
  }
}

// One 128 x SL_BN output tile at (m0, n0) of C = alpha A B + beta C.  Called by all
// SL_THREADS threads of the CTA; allocates and frees sl_tmem_cols<NST>() columns of tensor
// memory.  NST = 1 requires K <= SL_BK.
template <int NST>
__device__ __forceinline__ void sliced_tile(const TcArgs& g, int m0, int n0, uint8_t* smem) {
  constexpr uint32_t IDESC = idesc_tf32(SL_BN);
  constexpr uint32_t SL_TMEM_COLS = sl_tmem_cols<NST>();
  __shared__ uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  float* raw = reinterpret_cast<float*>(smem + NST * SL_STAGE);  // [NST][SL_RAW_FLOATS] staging
  float* scl = raw + NST * SL_RAW_FLOATS;  // [stage][TC_BM + SL_BN]: row scales of A, then of B
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wg = warp >> 2, wq = warp & 3;  // warpgroup, warp within it (its 32 TMEM lanes)

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(SL_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(&mbar[0]);
    mbar_init(&mbar[1]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t lane_base = tmem + ((uint32_t)(wq * 32) << 16) + (uint32_t)(wg * SL_HALF);
  const int row_l = wq * 32 + lane;  // this thread's row of the tile
  const int nvalid = g.N - n0 - wg * SL_HALF;

  float hi[SL_HALF], lo[SL_HALF];
#pragma unroll
  for (int j = 0; j < SL_HALF; ++j) hi[j] = lo[j] = 0.0f;
  const int nkb = NST == 1 ? (g.K > 0 ? 1 : 0) : (g.K + SL_BK - 1) / SL_BK;
  raw_prefetch<TC_BM>(g.A, g.sam, g.sak, m0, g.M, 0, g.K, raw);
  raw_prefetch<SL_BN>(g.B, g.sbn, g.sbk, n0, g.N, 0, g.K, raw + TC_BM * SL_RAW);
  cp_async_commit();
  uint32_t phase0 = 0, phase1 = 0;
  bool ok = true;
  for (int kb = 0; kb < nkb; ++kb) {
    const int s = NST == 1 ? 0 : (kb & 1);
    uint8_t* st = smem + s * SL_STAGE;
    float* rs = raw + s * SL_RAW_FLOATS;
    cp_async_wait_all();
    __syncthreads();  // block kb staged in rs; the other buffer was last read by the slicing of kb-1
    if (NST == 2 && kb + 1 < nkb) {  // next block's copies in flight during the slicing and the drain
      float* rn = raw + (s ^ 1) * SL_RAW_FLOATS;
      raw_prefetch<TC_BM>(g.A, g.sam, g.sak, m0, g.M, (kb + 1) * SL_BK, g.K, rn);
      raw_prefetch<SL_BN>(g.B, g.sbn, g.sbk, n0, g.N, (kb + 1) * SL_BK, g.K, rn + TC_BM * SL_RAW);
      cp_async_commit();
    }
    // stage s and tensor-memory buffer s were last used by block kb-2: its MMAs finished
    // and its levels were drained in the previous iteration, before the barrier above
    float* sc_s = scl + s * (TC_BM + SL_BN);
    slice_rows<TC_BM>(rs, st, st + SL_A_BYTES, st + 2 * SL_A_BYTES, sc_s);
    slice_rows<SL_BN>(rs + TC_BM * SL_RAW, st + 3 * SL_A_BYTES, st + 3 * SL_A_BYTES + SL_B_BYTES,
                      st + 3 * SL_A_BYTES + 2 * SL_B_BYTES, sc_s + TC_BM);
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(st), b0 = a0 + 3 * SL_A_BYTES;
      const uint32_t d0 = tmem + (uint32_t)(s * 3 * SL_BN);
#pragma unroll
      for (int kk = 0; kk < SL_BK / 8; ++kk) {
        const uint32_t off = kk * 256;  // two core matrices along K per MMA
        const uint64_t da0 = smem_desc(a0 + off, 128, 1024), da1 = smem_desc(a0 + SL_A_BYTES + off, 128, 1024),
                       da2 = smem_desc(a0 + 2 * SL_A_BYTES + off, 128, 1024);
        const uint64_t db0 = smem_desc(b0 + off, 128, 1024), db1 = smem_desc(b0 + SL_B_BYTES + off, 128, 1024),
                       db2 = smem_desc(b0 + 2 * SL_B_BYTES + off, 128, 1024);
        const uint32_t acc = kk > 0 ? 1u : 0u;
        mma_tf32(d0, da0, db0, IDESC, acc);                   // L0
        mma_tf32(d0 + SL_BN, da0, db1, IDESC, acc);           // L1
        mma_tf32(d0 + SL_BN, da1, db0, IDESC, 1u);
        mma_tf32(d0 + 2 * SL_BN, da0, db2, IDESC, acc);       // L2
        mma_tf32(d0 + 2 * SL_BN, da1, db1, IDESC, 1u);
        mma_tf32(d0 + 2 * SL_BN, da2, db0, IDESC, 1u);
      }
      mma_commit(&mbar[s]);
    }
    if (NST == 2 && kb > 0) {  // drain block kb-1 from buffer s^1 while block kb's MMAs run
      const int sp = s ^ 1;
      const bool w = sp == 0 ? mbar_wait(&mbar[0], phase0) : mbar_wait(&mbar[1], phase1);
      ok = __syncthreads_and(w);
      if (!ok) break;
      if (sp == 0) phase0 ^= 1; else phase1 ^= 1;
      tc_fence_after();
      const float* sp_s = scl + sp * (TC_BM + SL_BN);
      drain_levels(lane_base + (uint32_t)(sp * 3 * SL_BN), sp_s[row_l], sp_s + TC_BM + wg * SL_HALF, nvalid, hi,
                   lo);
      tc_fence_before();
    }
  }
  if (ok && nkb > 0) {
    const int sp = NST == 1 ? 0 : ((nkb - 1) & 1);
    const bool w = sp == 0 ? mbar_wait(&mbar[0], phase0) : mbar_wait(&mbar[1], phase1);
    ok = __syncthreads_and(w);
    if (ok) {
      tc_fence_after();
      const float* sp_s = scl + sp * (TC_BM + SL_BN);
      drain_levels(lane_base + (uint32_t)(sp * 3 * SL_BN), sp_s[row_l], sp_s + TC_BM + wg * SL_HALF, nvalid, hi,
                   lo);
    }
  }
  if (!ok) {
    // a wait expired: give the MMAs in flight a bounded chance to finish before the free
    mbar_wait(&mbar[0], phase0);
    if (NST == 2) mbar_wait(&mbar[1], phase1);
  }
  if (ok) {
    const int row = m0 + row_l;
    if (row < g.M) {
#pragma unroll
      for (int j = 0; j < SL_HALF; ++j) {
        const int col = n0 + wg * SL_HALF + j;
        if (col < g.N) {
          float* p = g.C + (int64_t)row * g.scm + (int64_t)col * g.scn;
          double v = g.alpha * ((double)hi[j] + (double)lo[j]);
          if (g.beta != 0.0) v += g.beta * (double)(*p);
          *p = (float)v;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(SL_TMEM_COLS)
                 : "memory");
  }
  if (!ok && tid == 0 && g.status) atomicOr(g.status, (unsigned)ST_TIMEOUT);
}

// A is short and B long: the tile covers 128 rows of M, so compute C^T = B^T A^T
__host__ __device__ __forceinline__ bool sliced_swap(int M, int N) { return M < 96 && N > M; }

__host__ __device__ __forceinline__ TcArgs sliced_args(int M, int N, int K, double alpha, const float* A,
                                                       int64_t sam, int64_t sak, const float* B, int64_t sbk,
                                                       int64_t sbn, double beta, float* C, int64_t scm,
                                                       int64_t scn, unsigned* status) {
  if (sliced_swap(M, N)) return TcArgs{N, M, K, alpha, beta, B, sbn, sbk, A, sak, sam, C, scn, scm, status};
  return TcArgs{M, N, K, alpha, beta, A, sam, sak, B, sbk, sbn, C, scm, scn, status};
}

template <int NST>
__global__ void __launch_bounds__(SL_THREADS, 3 - NST) gemm_sliced_kernel(TcArgs g) {
  extern __shared__ __align__(1024) uint8_t smem[];
  sliced_tile<NST>(g, blockIdx.y * TC_BM, blockIdx.x * SL_BN, smem);
}

// one CTA per tile of every job: prefix[j] = first tile of job j (tiles of the swapped
// problem when sliced_swap holds)
template <int NST>
__global__ void __launch_bounds__(SL_THREADS, 3 - NST)
    gemm_sliced_dense_kernel(const GemmJob<float, float, float>* __restrict__ jobs, const int* __restrict__ prefix,
                             int njobs, unsigned* status) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const int id = blockIdx.x;
  int lo = 0, hi = njobs;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (prefix[mid] <= id) lo = mid;
    else hi = mid;
  }
  // the job's arguments live in shared memory (uniform, read where used) rather than in
  // ~30 registers of every thread
  __shared__ TcArgs sg;
  if (threadIdx.x == 0) {
    const GemmJob<float, float, float> j = jobs[lo];
    sg = sliced_args(j.M, j.N, j.K, j.alpha, j.A, j.sam, j.sak, j.B, j.sbk, j.sbn, j.beta, j.C, j.scm, j.scn, status);
  }
  __syncthreads();
  const int local = id - prefix[lo];
  const int tn = (sg.N + SL_BN - 1) / SL_BN;
  sliced_tile<NST>(sg, (local / tn) * TC_BM, (local % tn) * SL_BN, smem);
}

template <int NST, typename K>
int sliced_configure(K kernel) {
  static std::atomic<int> configured{-1};
  int dev = 0;
  TT_CUDA_CHECK(cudaGetDevice(&dev));
  if (configured != dev) {
    TT_CUDA_CHECK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sl_smem<NST>()));
    configured = dev;
  }
  return TT_OK;
}
}  // namespace

int gemm_tf32x3(cudaStream_t s, int M, int N, int K, double alpha, const float* A, int64_t sam,
                int64_t sak, const float* B, int64_t sbk, int64_t sbn, double beta, float* C,
                int64_t scm, int64_t scn, unsigned* status, bool acc64) {
  if (M <= 0 || N <= 0) return TT_OK;
  if (K <= 0) return gemm<float, float, float>(s, M, N, K, alpha, A, sam, sak, B, sbk, sbn, beta, C, scm, scn);
  // a tile is 128 rows of M: if M is short and N long, compute C^T = B^T A^T instead
  if (M < 96 && N > M) {
    std::swap(M, N);
    std::swap(A, B);
    const int64_t t_sam = sbn, t_sak = sbk, t_sbk = sak, t_sbn = sam;
    sam = t_sam;
    sak = t_sak;
    sbk = t_sbk;
    sbn = t_sbn;
    std::swap(scm, scn);
  }
  TcArgs a{M, N, K, alpha, beta, A, sam, sak, B, sbk, sbn, C, scm, scn, status};
  if (acc64) return launch_tc<64, double>(s, a);
  if (N <= 64) return launch_tc<64, float>(s, a);
  return launch_tc<128, float>(s, a);
}


int64_t sliced_tiles(int M, int N) {
  if (M <= 0 || N <= 0) return 0;
  if (sliced_swap(M, N)) std::swap(M, N);
  return ceil_div(M, TC_BM) * ceil_div(N, SL_BN);
}

int gemm_sliced(cudaStream_t s, int M, int N, int K, double alpha, const float* A, int64_t sam, int64_t sak,
                const float* B, int64_t sbk, int64_t sbn, double beta, float* C, int64_t scm, int64_t scn,
                unsigned* status) {
  if (M <= 0 || N <= 0) return TT_OK;
  if (K <= 0) return gemm<float, float, float>(s, M, N, K, alpha, A, sam, sak, B, sbk, sbn, beta, C, scm, scn);
  const TcArgs a = sliced_args(M, N, K, alpha, A, sam, sak, B, sbk, sbn, beta, C, scm, scn, status);
  dim3 grid((unsigned)ceil_div(a.N, SL_BN), (unsigned)ceil_div(a.M, TC_BM));
  if (grid.y > 65535u) return fail(TT_ERR_UNSUPPORTED, "gemm_sliced: M too large");
  if (K <= SL_BK) {
    TT_TRY(sliced_configure<1>(gemm_sliced_kernel<1>));
    gemm_sliced_kernel<1><<<grid, SL_THREADS, sl_smem<1>(), s>>>(a);
  } else {
    TT_TRY(sliced_configure<2>(gemm_sliced_kernel<2>));
    gemm_sliced_kernel<2><<<grid, SL_THREADS, sl_smem<2>(), s>>>(a);
  }
  TT_LAUNCH_CHECK();
  return TT_OK;
}

int gemm_sliced_dense(cudaStream_t s, int njobs, const GemmJob<float, float, float>* d_jobs, const int* d_prefix,
                      int64_t total_tiles, int K_max, unsigned* status) {
  if (njobs <= 0 || total_tiles <= 0) return TT_OK;
  if (total_tiles > 0x7fffffff) return fail(TT_ERR_UNSUPPORTED, "gemm_sliced_dense: too many tiles");
  const unsigned g = (unsigned)total_tiles;
  if (K_max <= SL_BK) {
    TT_TRY(sliced_configure<1>(gemm_sliced_dense_kernel<1>));
    gemm_sliced_dense_kernel<1><<<g, SL_THREADS, sl_smem<1>(), s>>>(d_jobs, d_prefix, njobs, status);
  } else {
    TT_TRY(sliced_configure<2>(gemm_sliced_dense_kernel<2>));
    gemm_sliced_dense_kernel<2><<<g, SL_THREADS, sl_smem<2>(), s>>>(d_jobs, d_prefix, njobs, status);
  }
  TT_LAUNCH_CHECK();
  return TT_OK;
}

}  // namespace tt
