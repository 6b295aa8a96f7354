// FP64 instantiations of the fused sweep kernel for K equal to the lane count (K = 4, 8, 16, 32;
// g4 on the affine set, eq. 10): the class strides are compile-time constants.
#include "launch.h"

namespace sgs {
template <typename T>
cudaError_t launch_sweep_keq(const SweepArgs<T>& a, int M, int G, bool diag, int tiles,
                             size_t smem, cudaStream_t st) {
  return launch_sweep_variant<T, false, true>(a, M, G, diag, tiles, smem, st);
}
template <typename T>
cudaError_t prepare_sweep_keq(int M, int G, size_t smem, size_t smem_diag) {
  return prepare_sweep_variant<T, false, true>(M, G, smem, smem_diag);
}
template cudaError_t prepare_sweep_keq<double>(int, int, size_t, size_t);
template cudaError_t launch_sweep_keq<double>(const SweepArgs<double>&, int, int, bool, int, size_t,
                                         cudaStream_t);
}  // namespace sgs
