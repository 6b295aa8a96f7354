// Instantiation and launch of the MLR class-model kernel (tensor cores), FP32 and FP64 output.
#include "mlr.cuh"

namespace sgs {

template <typename T>
struct MlrGrant {
  static SmemGrants g;
};
template <typename T> SmemGrants MlrGrant<T>::g;

template <typename T>
cudaError_t launch_mlr(const MlrArgs& a, cudaStream_t st) {
  const size_t smem = mlr_smem_bytes(a.d, a.dpad, a.npad, a.K);
  const cudaError_t e = grant_smem(k_mlr<T>, smem, MlrGrant<T>::g);
  if (e != cudaSuccess) return e;
  const int grid = (a.n + MLR_TILE - 1) / MLR_TILE;
  k_mlr<T><<<grid, MLR_THREADS, smem, st>>>(a);
  return cudaGetLastError();
}

template cudaError_t launch_mlr<float>(const MlrArgs&, cudaStream_t);
template cudaError_t launch_mlr<double>(const MlrArgs&, cudaStream_t);

}  // namespace sgs
