// Instantiations and launchers of the reverse-pass kernels (FP32 and FP64).
#include "adjoint.cuh"

namespace sgs {

template <typename T, int M>
static cudaError_t vjp_g(const AdjArgs<T>& a, int G, int blocks, cudaStream_t st) {
  switch (G) {
    case 4: k_adj_vjp<T, M, 4><<<blocks, ADJ_THREADS, 0, st>>>(a); break;
    case 8: k_adj_vjp<T, M, 8><<<blocks, ADJ_THREADS, 0, st>>>(a); break;
    case 16: k_adj_vjp<T, M, 16><<<blocks, ADJ_THREADS, 0, st>>>(a); break;
    case 32: k_adj_vjp<T, M, 32><<<blocks, ADJ_THREADS, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adj_vjp(const AdjArgs<T>& a, int M, int G, int blocks, cudaStream_t st) {
  switch (M) {
    case 0: return vjp_g<T, 0>(a, G, blocks, st);
    case 1: return vjp_g<T, 1>(a, G, blocks, st);
    case 2: return vjp_g<T, 2>(a, G, blocks, st);
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_adj_gt(AdjShape s, int M, const T* v_loc, const T* v_2, const T* omega,
                          T* zbar, cudaStream_t st) {
  const int blocks = (int)(((size_t)s.n * s.K + ADJ_THREADS - 1) / ADJ_THREADS);
  switch (M) {
    case 0: k_adj_gt<T, 0><<<blocks, ADJ_THREADS, 0, st>>>(s, v_loc, v_2, omega, zbar); break;
    case 1: k_adj_gt<T, 1><<<blocks, ADJ_THREADS, 0, st>>>(s, v_loc, v_2, omega, zbar); break;
    case 2: k_adj_gt<T, 2><<<blocks, ADJ_THREADS, 0, st>>>(s, v_loc, v_2, omega, zbar); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adj_init(AdjShape s, int G, const T* p, const T* zbar, T* glogp,
                            cudaStream_t st) {
  const int blocks = (s.n + ADJ_THREADS / G - 1) / (ADJ_THREADS / G);
  switch (G) {
    case 4: k_adj_init<T, 4><<<blocks, ADJ_THREADS, 0, st>>>(s, p, zbar, glogp); break;
    case 8: k_adj_init<T, 8><<<blocks, ADJ_THREADS, 0, st>>>(s, p, zbar, glogp); break;
    case 16: k_adj_init<T, 16><<<blocks, ADJ_THREADS, 0, st>>>(s, p, zbar, glogp); break;
    case 32: k_adj_init<T, 32><<<blocks, ADJ_THREADS, 0, st>>>(s, p, zbar, glogp); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_exp_logp(AdjShape s, int G, const T* logp, T* p, cudaStream_t st) {
  const int blocks = (s.n + ADJ_THREADS / G - 1) / (ADJ_THREADS / G);
  switch (G) {
    case 4: k_exp_logp<T, 4><<<blocks, ADJ_THREADS, 0, st>>>(s, logp, p); break;
    case 8: k_exp_logp<T, 8><<<blocks, ADJ_THREADS, 0, st>>>(s, logp, p); break;
    case 16: k_exp_logp<T, 16><<<blocks, ADJ_THREADS, 0, st>>>(s, logp, p); break;
    case 32: k_exp_logp<T, 32><<<blocks, ADJ_THREADS, 0, st>>>(s, logp, p); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// One block per column of the partials; each thread adds a strided set of rows, then the warps'
// shuffle sums in warp order: the same inputs always give the same bits.
__global__ void __launch_bounds__(ADJ_THREADS) k_adj_sum(const double* part, int blocks,
                                                          double* acc) {
  __shared__ double red[ADJ_THREADS / 32];
  const double* col = part + (size_t)blockIdx.x * blocks;
  double t = 0.0;
  for (int r = threadIdx.x; r < blocks; r += ADJ_THREADS) t += col[r];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < ADJ_THREADS / 32; ++w) s += red[w];
    acc[blockIdx.x] += s;
  }
}

cudaError_t launch_adj_sum(const double* part, int blocks, int np, double* acc, cudaStream_t st) {
  if (np < 1 || blocks < 1) return cudaErrorInvalidValue;
  k_adj_sum<<<np, ADJ_THREADS, 0, st>>>(part, blocks, acc);
  return cudaGetLastError();
}

#define SGS_ADJ_INST(T)                                                                       \
  template cudaError_t launch_adj_vjp<T>(const AdjArgs<T>&, int, int, int, cudaStream_t);     \
  template cudaError_t launch_adj_gt<T>(AdjShape, int, const T*, const T*, const T*, T*,      \
                                        cudaStream_t);                                        \
  template cudaError_t launch_adj_init<T>(AdjShape, int, const T*, const T*, T*, cudaStream_t); \
  template cudaError_t launch_exp_logp<T>(AdjShape, int, const T*, T*, cudaStream_t);
SGS_ADJ_INST(float)
SGS_ADJ_INST(double)
#undef SGS_ADJ_INST

}  // namespace sgs
