// Launch entry points of the fused sweep, compiled in their own translation units per
// precision so that the build runs in parallel.
#pragma once

#include <cuda_runtime.h>

#include "sweep.cuh"

namespace sgs {

template <typename T>
cudaError_t launch_sweep(const SweepArgs<T>& a, int M, int G, bool diag, int tiles, size_t smem,
                         cudaStream_t st);

// Grant the dynamic shared memory of the plain and traced variants before any launch (so
// that graph capture never changes kernel attributes).
template <typename T>
cudaError_t prepare_sweep(int M, int G, size_t smem, size_t smem_diag);

// The same for K equal to the lane count G and full-width tiles (NC = 256 / G): compile-time
// class strides and z-tile stride.
template <typename T>
cudaError_t launch_sweep_keq(const SweepArgs<T>& a, int M, int G, bool diag, int tiles,
                             size_t smem, cudaStream_t st);
template <typename T>
cudaError_t prepare_sweep_keq(int M, int G, size_t smem, size_t smem_diag);

// The same with g4 as the probability simplex indicator.
template <typename T>
cudaError_t launch_sweep_simplex(const SweepArgs<T>& a, int M, int G, bool diag, int tiles,
                                 size_t smem, cudaStream_t st);
template <typename T>
cudaError_t prepare_sweep_simplex(int M, int G, size_t smem, size_t smem_diag);

extern template cudaError_t prepare_sweep_simplex<float>(int, int, size_t, size_t);
extern template cudaError_t prepare_sweep_simplex<double>(int, int, size_t, size_t);
extern template cudaError_t launch_sweep_simplex<float>(const SweepArgs<float>&, int, int, bool,
                                                        int, size_t, cudaStream_t);
extern template cudaError_t launch_sweep_simplex<double>(const SweepArgs<double>&, int, int, bool,
                                                         int, size_t, cudaStream_t);
extern template cudaError_t prepare_sweep_keq<float>(int, int, size_t, size_t);
extern template cudaError_t prepare_sweep_keq<double>(int, int, size_t, size_t);
extern template cudaError_t launch_sweep_keq<float>(const SweepArgs<float>&, int, int, bool, int,
                                                    size_t, cudaStream_t);
extern template cudaError_t launch_sweep_keq<double>(const SweepArgs<double>&, int, int, bool,
                                                     int, size_t, cudaStream_t);
extern template cudaError_t prepare_sweep<float>(int, int, size_t, size_t);
extern template cudaError_t prepare_sweep<double>(int, int, size_t, size_t);
extern template cudaError_t launch_sweep<float>(const SweepArgs<float>&, int, int, bool, int,
                                                size_t, cudaStream_t);
extern template cudaError_t launch_sweep<double>(const SweepArgs<double>&, int, int, bool, int,
                                                 size_t, cudaStream_t);

}  // namespace sgs
