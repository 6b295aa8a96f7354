// Device helpers shared by the SegSALSA-STR kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

namespace sgs {

template <typename T> struct CplxOf;
template <> struct CplxOf<float> { using type = float2; };
template <> struct CplxOf<double> { using type = double2; };
template <typename T> using cplx = typename CplxOf<T>::type;

template <typename T> __host__ __device__ __forceinline__ cplx<T> mkc(T x, T y) {
  cplx<T> r; r.x = x; r.y = y; return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
template <typename C> __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {
  C r; r.x = a.x * b.x + a.y * b.y; r.y = a.y * b.x - a.x * b.y; return r;
}
// multiply by -i (forward) or +i (inverse)
template <typename C> __device__ __forceinline__ C cmul_mi(C a) { C r; r.x = a.y; r.y = -a.x; return r; }
template <typename C> __device__ __forceinline__ C cmul_pi(C a) { C r; r.x = -a.y; r.y = a.x; return r; }

// Sum over aligned groups of G lanes (G a power of two <= 32); every lane of the warp must
// call it. All G lanes of a group receive the group total.
template <int G, typename T> __device__ __forceinline__ T group_sum(T v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, G);
  return v;
}

// ------------------------------------------------------------ async copies and mbarriers
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Per-thread asynchronous 4- or 8-byte copy global -> shared; valid == false fills zeros.
template <int BYTES>
__device__ __forceinline__ void cp_async_zfill(void* dst, const void* src, bool valid) {
  const int n = valid ? BYTES : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(smem_addr(dst)), "l"(src),
               "n"(BYTES), "r"(n)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
// Bulk (TMA engine) copy of `bytes` (multiple of 16, both addresses 16-byte aligned) from
// global to this CTA's shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase with `parity` to complete, giving up after ~`budget` clock cycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  long long budget) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > budget) return false;
  return true;
}
constexpr long long WAIT_BUDGET_CYCLES = 2000000000LL;  // about one second at 2 GHz

// Programmatic dependent launch: a kernel launched with the programmatic-serialization
// attribute may start before its predecessor in the stream has finished; it must call
// pdl_wait() before touching anything the predecessor writes (the wait returns once the
// predecessor grid has completed and its memory is visible). pdl_trigger() lets the next
// kernel start its own independent prologue. Both are no-ops for ordinary launches.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

// Launch with the programmatic-serialization attribute (see pdl_wait).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// Identity of the calling thread's current CUDA context: unique for the life of the process, so
// it changes when a device is reset and its primary context is created anew. 0 when it cannot
// be read (no current context, or a driver without cuCtxGetId).
inline unsigned long long current_context_id() {
  using Fn = int (*)(void*, unsigned long long*);  // CUresult cuCtxGetId(CUcontext, id*)
  static const Fn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<Fn>(f);
  }();
  unsigned long long id = 0;
  if (!fn || fn(nullptr, &id) != 0) return 0;
  return id;
}

// Dynamic shared memory granted to one kernel, per device and per context: the attribute set
// by cudaFuncSetAttribute belongs to the current device's context, so a second GPU (or a
// context created after a device reset) starts from nothing.
constexpr int kMaxDevices = 64;
struct SmemGrants {
  std::mutex mu;
  unsigned long long ctx[kMaxDevices] = {};
  size_t bytes[kMaxDevices] = {};
};

// Raise `kern`'s dynamic shared-memory limit on the current device to at least `smem`.
template <typename K>
inline cudaError_t grant_smem(K kern, size_t smem, SmemGrants& g) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  const unsigned long long ctx = current_context_id();
  std::lock_guard<std::mutex> lk(g.mu);
  if (g.ctx[dev] != ctx) {
    g.ctx[dev] = ctx;
    g.bytes[dev] = 0;
  }
  if (smem <= g.bytes[dev] && ctx != 0) return cudaSuccess;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && smem > g.bytes[dev]) g.bytes[dev] = smem;
  return e;
}

__host__ __device__ __forceinline__ int wrap_idx(int v, int n) {
  int r = v % n;
  return r < 0 ? r + n : r;
}

// Deterministic block-wide sum of a double (blockDim.x a multiple of 32, <= 1024).
__device__ __forceinline__ double block_sum_d(double v, double* red32) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red32[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    const int nw = (blockDim.x + 31) >> 5;
    t = (l < nw) ? red32[l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;  // valid in thread 0
}

__device__ __forceinline__ double block_min_d(double v, double* red32) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red32[w] = v;
  __syncthreads();
  double t = 1e300;
  if (threadIdx.x < 32) {
    const int nw = (blockDim.x + 31) >> 5;
    t = (l < nw) ? red32[l] : 1e300;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = fmin(t, __shfl_xor_sync(0xffffffffu, t, o));
  }
  return t;
}

__device__ __forceinline__ double block_max_d(double v, double* red32) {
  return -block_min_d(-v, red32);
}

// Block reductions of per-thread values in the working precision T: shuffles in T within each
// warp, then thread 0 adds (or compares) the warp results in FP64 in warp order. The FP64 work is
// one operation per warp (FP64 is a narrow pipe on this part); the order is fixed, so equal
// inputs give equal bits. The result is valid in thread 0.
template <typename T>
__device__ __forceinline__ double block_sum_w(T v, double* red32) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red32[w] = (double)v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)((blockDim.x + 31) >> 5); ++i) t += red32[i];
  return t;
}
template <typename T>
__device__ __forceinline__ double block_min_w(T v, double* red32) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red32[w] = (double)v;
  __syncthreads();
  double t = 1e300;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)((blockDim.x + 31) >> 5); ++i) t = fmin(t, red32[i]);
  return t;
}
template <typename T>
__device__ __forceinline__ double block_max_w(T v, double* red32) {
  return -block_min_w<T>(-v, red32);
}

}  // namespace sgs
