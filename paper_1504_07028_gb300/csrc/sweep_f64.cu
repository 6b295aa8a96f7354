// FP64 instantiations of the fused sweep kernel.
#include "launch.h"

namespace sgs {
template <typename T>
cudaError_t launch_sweep(const SweepArgs<T>& a, int M, int G, bool diag, int tiles, size_t smem,
                         cudaStream_t st) {
  return diag ? launch_sweep_md<T, true>(a, M, G, tiles, smem, st)
              : launch_sweep_md<T, false>(a, M, G, tiles, smem, st);
}
template cudaError_t launch_sweep<double>(const SweepArgs<double>&, int, int, bool, int, size_t,
                                         cudaStream_t);
}  // namespace sgs
