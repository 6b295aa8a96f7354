// Launch entry points of the fused sweep, compiled in their own translation units per
// precision so that the build runs in parallel.
#pragma once

#include <cuda_runtime.h>

#include "sweep.cuh"

namespace sgs {

template <typename T>
cudaError_t launch_sweep(const SweepArgs<T>& a, int M, int G, bool diag, int tiles, size_t smem,
                         cudaStream_t st);

extern template cudaError_t launch_sweep<float>(const SweepArgs<float>&, int, int, bool, int,
                                                size_t, cudaStream_t);
extern template cudaError_t launch_sweep<double>(const SweepArgs<double>&, int, int, bool, int,
                                                 size_t, cudaStream_t);

}  // namespace sgs
