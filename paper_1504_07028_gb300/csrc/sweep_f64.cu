// FP64 instantiations of the fused sweep kernel (g4 on the affine set, eq. 10).
#include "launch.h"

namespace sgs {
template <typename T>
cudaError_t launch_sweep(const SweepArgs<T>& a, int M, int G, bool diag, int tiles, size_t smem,
                         cudaStream_t st) {
  return launch_sweep_variant<T, false, false>(a, M, G, diag, tiles, smem, st);
}
template <typename T>
cudaError_t prepare_sweep(int M, int G, size_t smem, size_t smem_diag) {
  return prepare_sweep_variant<T, false, false>(M, G, smem, smem_diag);
}
template cudaError_t prepare_sweep<double>(int, int, size_t, size_t);
template cudaError_t launch_sweep<double>(const SweepArgs<double>&, int, int, bool, int, size_t,
                                      cudaStream_t);
}  // namespace sgs
