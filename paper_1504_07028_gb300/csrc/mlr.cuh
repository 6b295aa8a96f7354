// Class model of the experiments (Sec. 5): the class probabilities p_i that enter problem (7)
// come from a multinomial logistic regression on the d-band spectra,
//     p_i = softmax_k(w_k^T x_i + b_k),
// a dense n x d x K contraction followed by a per-pixel softmax. The contraction runs on the
// 5th-generation tensor cores: one CTA per tile of 128 pixels stages the spectra (A, 128 x dpad)
// and the weights (B, Npad x dpad) as BF16 in shared memory in the K-major, no-swizzle
// core-matrix layout, one thread issues tcgen05.mma (kind::f16, M = 128, N = Npad, K = 16 per
// instruction) into an FP32 accumulator in tensor memory, and every warp reads its 32 rows
// back with tcgen05.ld for the bias + softmax epilogue in FP32.
#pragma once

#include <stdint.h>

#include "common.cuh"

namespace sgs {

constexpr int MLR_TILE = 128;     // pixels per CTA (the MMA's M)
constexpr int MLR_MAXD = 256;     // most spectral bands
constexpr int MLR_THREADS = 128;  // four warps: warp w owns accumulator lanes 32w .. 32w+31
constexpr int MLR_TMEM_COLS = 32; // allocation granularity (holds N <= 32 FP32 columns)

struct MlrArgs {
  const uint16_t* x;   // [n][d] BF16 bit patterns, pixel-major
  const uint16_t* w;   // [K][d] BF16 bit patterns
  const float* bias;   // [K] or nullptr
  void* p;             // [n][K] output in the handle's precision
  int* err;            // set when a bounded wait gives up
  int n, d, dpad, K, npad;
  long long budget;    // clock cycles a bounded wait may take
  uint32_t probe;      // extra bytes armed on the staging barrier (0; 16 in the wait test)
};

// Byte offset of element (r, k) in a K-major, no-swizzle operand tile with kc = dpad / 8
// core-matrix columns: core matrix (r / 8, k / 8) is 128 contiguous bytes (8 rows of 16 bytes)
// and the core matrices of one 8-row group follow each other along k.
__device__ __forceinline__ uint32_t mlr_canon_off(int r, int k, int kc) {
  return (uint32_t)((((r >> 3) * kc + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

// Shared-memory matrix descriptor (no swizzle): start address, leading byte offset (between
// core matrices adjacent along K), stride byte offset (between 8-row groups), descriptor
// version 1 in bits 46-47.
__device__ __forceinline__ uint64_t mlr_smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A and B
// (bits 7-9 and 10-12 = 1), both K-major, N / 8 in bits 17-22, M / 16 in bits 24-28.
__host__ __device__ constexpr uint32_t mlr_idesc(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                   smem_addr(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}
// Generic-proxy shared-memory writes become visible to the tensor core (async proxy).
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void tc_mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                            uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrive on `bar` once every tcgen05.mma this thread issued has completed.
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
          smem_addr(bar))
      : "memory");
}
// 16 consecutive FP32 columns of this thread's accumulator lane.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Dynamic shared memory of a CTA: the A and B operand tiles, the barriers and the TMEM slot,
// then the staging areas the tile's spectra (128 rows of d values) and the weights (K rows)
// arrive in as laid out in memory.
__host__ __device__ inline size_t mlr_stage_a_offset(int dpad, int npad) {
  return (size_t)(MLR_TILE + npad) * dpad * 2 + 64;
}
__host__ __device__ inline size_t mlr_stage_b_offset(int d, int dpad, int npad) {
  return mlr_stage_a_offset(dpad, npad) + ((size_t)MLR_TILE * d * 2 + 15) / 16 * 16;
}
inline size_t mlr_smem_bytes(int d, int dpad, int npad, int K) {
  return mlr_stage_b_offset(d, dpad, npad) + ((size_t)K * d * 2 + 15) / 16 * 16;
}

// Copy `bytes` from global src (16-byte aligned) to shared dst: the 16-byte multiple by one
// bulk copy issued by thread 0 (counted into `tx`), the rest by plain loads of all threads.
__device__ __forceinline__ void mlr_stage_run(unsigned char* dst, const unsigned char* src,
                                              uint32_t bytes, uint64_t* bar) {
  const uint32_t bulk = bytes & ~15u;
  if (threadIdx.x == 0 && bulk) bulk_g2s(dst, src, bulk, bar);
  for (uint32_t i = bulk + threadIdx.x; i < bytes; i += MLR_THREADS) dst[i] = __ldg(src + i);
}

// Thread r packs row r of a row-major staged matrix (rows of d BF16 values) into the
// K-major core-matrix layout, 16 bytes (8 bands) per store; rows >= rows_valid and bands >= d
// are zero.
__device__ __forceinline__ void mlr_pack_row(unsigned char* dst, const unsigned char* staged,
                                             int r, int rows_valid, int d, int kc) {
  const uint16_t* srow = reinterpret_cast<const uint16_t*>(staged) + (size_t)r * d;
  const bool rv = r < rows_valid;
  for (int c = 0; c < kc; ++c) {
    uint32_t w4[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int k0 = 8 * c + 2 * e;
      const uint32_t lo = (rv && k0 < d) ? srow[k0] : 0u;
      const uint32_t hi = (rv && k0 + 1 < d) ? srow[k0 + 1] : 0u;
      w4[e] = lo | (hi << 16);
    }
    *reinterpret_cast<uint4*>(dst + mlr_canon_off(r, 8 * c, kc)) = make_uint4(w4[0], w4[1], w4[2], w4[3]);
  }
}

template <typename T>
__global__ void __launch_bounds__(MLR_THREADS) k_mlr(const MlrArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* As = smem_raw;
  unsigned char* Bs = As + (size_t)MLR_TILE * a.dpad * 2;
  uint64_t* bar = reinterpret_cast<uint64_t*>(Bs + (size_t)a.npad * a.dpad * 2);
  uint64_t* lbar = bar + 1;                      // completion of the staging copies
  uint32_t* slot = reinterpret_cast<uint32_t*>(bar + 2);
  unsigned char* stA = smem_raw + mlr_stage_a_offset(a.dpad, a.npad);
  unsigned char* stB = smem_raw + mlr_stage_b_offset(a.d, a.dpad, a.npad);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kc = a.dpad >> 3;
  const int row0 = blockIdx.x * MLR_TILE;
  const int rows = min(MLR_TILE, a.n - row0);
  // the tile's spectra are one contiguous run of rows * d values starting at byte
  // row0 * d * 2 (a multiple of 256) of the 16-byte aligned x; the weights likewise
  const uint32_t bytesA = (uint32_t)rows * a.d * 2, bytesB = (uint32_t)a.K * a.d * 2;
  const unsigned char* srcA = reinterpret_cast<const unsigned char*>(a.x + (size_t)row0 * a.d);
  const unsigned char* srcB = reinterpret_cast<const unsigned char*>(a.w);

  if (warp == 0) tmem_alloc(slot, MLR_TMEM_COLS);
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    mbar_init(lbar, 1);
    mbar_fence_init();
    mbar_arrive_expect_tx(lbar, (bytesA & ~15u) + (bytesB & ~15u) + a.probe);
  }
  mlr_stage_run(stA, srcA, bytesA, lbar);
  mlr_stage_run(stB, srcB, bytesB, lbar);
  __syncthreads();                                // barrier init and the tail bytes
  const bool staged = mbar_wait_bounded(lbar, 0, a.budget);
  if (!staged) {
    // report, and give the staging copies in flight a second bounded chance to land before
    // the buffers are overwritten below (the tile is then computed from zeros and discarded)
    if (threadIdx.x == 0) atomicExch(a.err, 1);
    mbar_wait_bounded(lbar, 0, a.budget);
  }
  mlr_pack_row(As, stA, threadIdx.x, staged ? rows : 0, a.d, kc);
  if (threadIdx.x < a.npad) mlr_pack_row(Bs, stB, threadIdx.x, staged ? a.K : 0, a.d, kc);
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *slot;

  if (threadIdx.x == 0) {
    const uint32_t idesc = mlr_idesc(MLR_TILE, a.npad);
    const uint32_t sa = smem_addr(As), sb = smem_addr(Bs);
    // K step s covers bands 16s .. 16s+15 = core-matrix columns 2s, 2s+1
    for (int s = 0; s < a.dpad / 16; ++s) {
      const uint64_t ad = mlr_smem_desc(sa + s * 256, 128, kc * 128);
      const uint64_t bd = mlr_smem_desc(sb + s * 256, 128, kc * 128);
      tc_mma_bf16(tbase, ad, bd, idesc, s > 0 ? 1u : 0u);
    }
    tc_commit(bar);
  }
  const bool ok = mbar_wait_bounded(bar, 0, a.budget);
  tc_fence_after();
  if (!ok) {
    // report, and give the MMA a second bounded chance to finish. A CTA has to release its
    // tensor memory before it exits, so it is freed below either way; the error flag marks
    // the launch's output as invalid (the call returns SEGSALSA_ERR_TIMEOUT and keeps p)
    if (threadIdx.x == 0) atomicExch(a.err, 1);
    mbar_wait_bounded(bar, 0, a.budget);
  } else {
    // epilogue: thread (warp w, lane l) holds the logits of tile row 32w + l
    float lg[32];
    const uint32_t taddr = tbase + ((uint32_t)(warp * 32) << 16);
    tc_ld16(taddr, lg);
    if (a.npad > 16) tc_ld16(taddr + 16, lg + 16);
    const int row = row0 + warp * 32 + lane;
    if (row < a.n) {
      float m = -INFINITY;
#pragma unroll
      for (int k = 0; k < 32; ++k)
        if (k < a.K) {
          lg[k] += a.bias ? a.bias[k] : 0.f;
          m = fmaxf(m, lg[k]);
        }
      float s = 0.f;
#pragma unroll
      for (int k = 0; k < 32; ++k)
        if (k < a.K) {
          lg[k] = expf(lg[k] - m);
          s += lg[k];
        }
      const float inv = 1.f / s;
      T* out = reinterpret_cast<T*>(a.p) + (size_t)row * a.K;
#pragma unroll
      for (int k = 0; k < 32; ++k)
        if (k < a.K) out[k] = (T)(lg[k] * inv);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tbase, MLR_TMEM_COLS);
}

template <typename T>
cudaError_t launch_mlr(const MlrArgs& a, cudaStream_t st);

}  // namespace sgs
