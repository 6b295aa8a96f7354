// FP32 instantiations of the row-transform and column-solve passes.
#define SGS_FFT_INSTANTIATE
#include "zfused.cuh"

namespace sgs {
template cudaError_t launch_row<float>(bool, const RowArgs<float>&, dim3, const RowLaunch&, cudaStream_t, bool);
template cudaError_t launch_col<float>(const ColArgs<float>&, int, int, size_t, cudaStream_t);
template cudaError_t prepare_fft<float>(const RowLaunch&, size_t);
template cudaError_t launch_row_pipe<float>(bool, const RowArgs<float>&, int, size_t, cudaStream_t);
template cudaError_t row_pipe_blocks_per_sm<float>(bool, size_t, int*);
template cudaError_t launch_row_p2<float>(bool, const RowArgs<float>&, dim3, size_t, cudaStream_t);
template cudaError_t launch_zfused<float>(const ZfArgs<float>&, int, int, size_t, cudaStream_t);
template int zfused_max_clusters<float>(int, int, size_t);
template cudaError_t launch_zseq<float>(const ZseqArgs<float>&, int, int, size_t, cudaStream_t, int*);

}  // namespace sgs
