// FP64 instantiations of the fused sweep kernel with g4 read as the probability
// simplex indicator (the variant of Sec. 4's description of the MPO of g4).
#include "launch.h"

namespace sgs {
template <typename T>
cudaError_t launch_sweep_simplex(const SweepArgs<T>& a, int M, int G, bool diag, int tiles,
                                 size_t smem, cudaStream_t st) {
  return launch_sweep_variant<T, true, false>(a, M, G, diag, tiles, smem, st);
}
template <typename T>
cudaError_t prepare_sweep_simplex(int M, int G, size_t smem, size_t smem_diag) {
  return prepare_sweep_variant<T, true, false>(M, G, smem, smem_diag);
}
template cudaError_t prepare_sweep_simplex<double>(int, int, size_t, size_t);
template cudaError_t launch_sweep_simplex<double>(const SweepArgs<double>&, int, int, bool, int,
                                              size_t, cudaStream_t);
}  // namespace sgs
