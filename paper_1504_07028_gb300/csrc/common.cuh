// Device helpers shared by the SegSALSA-STR kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

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

}  // namespace sgs
