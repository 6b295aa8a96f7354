// FP64 instantiations of the fused sweep kernel.
#include "launch.h"

namespace sgs {
template <typename T>
cudaError_t launch_sweep(const SweepArgs<T>& a, int M, int G, bool diag, int tiles, size_t smem,
                         cudaStream_t st) {
  return diag ? launch_sweep_md<T, true>(a, M, G, tiles, smem, st)
              : launch_sweep_md<T, false>(a, M, G, tiles, smem, st);
}
template <typename T>
cudaError_t prepare_sweep(int M, int G, size_t smem, size_t smem_diag) {
#define SGS_PREP(MM, GG) \
  if (M == MM && G == GG) return prepare_sweep_inst<T, MM, GG>(smem, smem_diag);
  SGS_PREP(0, 4) SGS_PREP(0, 8) SGS_PREP(0, 16) SGS_PREP(0, 32)
  SGS_PREP(1, 4) SGS_PREP(1, 8) SGS_PREP(1, 16) SGS_PREP(1, 32)
  SGS_PREP(2, 4) SGS_PREP(2, 8) SGS_PREP(2, 16) SGS_PREP(2, 32)
#undef SGS_PREP
  return cudaErrorInvalidValue;
}
template cudaError_t prepare_sweep<double>(int, int, size_t, size_t);
template cudaError_t launch_sweep<double>(const SweepArgs<double>&, int, int, bool, int, size_t,
                                         cudaStream_t);
}  // namespace sgs
