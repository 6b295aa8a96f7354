// Instantiation and launch of the MLR class-model kernel (tensor cores), FP32 and FP64 output.
#include "mlr.cuh"

namespace sgs {

template <typename T>
struct MlrGrant {
  static size_t g;
};
template <typename T> size_t MlrGrant<T>::g = 0;

template <typename T>
cudaError_t launch_mlr(const MlrArgs& a, cudaStream_t st) {
  const size_t smem = mlr_smem_bytes(a.d, a.dpad, a.npad, a.K);
  if (smem > MlrGrant<T>::g) {
    const cudaError_t e =
        cudaFuncSetAttribute(k_mlr<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    MlrGrant<T>::g = smem;
  }
  const int grid = (a.n + MLR_TILE - 1) / MLR_TILE;
  k_mlr<T><<<grid, MLR_THREADS, smem, st>>>(a);
  return cudaGetLastError();
}

template cudaError_t launch_mlr<float>(const MlrArgs&, cudaStream_t);
template cudaError_t launch_mlr<double>(const MlrArgs&, cudaStream_t);

}  // namespace sgs
