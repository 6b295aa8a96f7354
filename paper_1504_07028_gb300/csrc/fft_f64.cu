// FP64 instantiations of the row-transform and column-solve passes.
#define SGS_FFT_INSTANTIATE
#include "zfused.cuh"

namespace sgs {
template cudaError_t launch_row<double>(bool, const RowArgs<double>&, dim3, const RowLaunch&, cudaStream_t, bool);
template cudaError_t launch_col<double>(const ColArgs<double>&, int, int, size_t, cudaStream_t);
template cudaError_t prepare_fft<double>(const RowLaunch&, size_t);
template cudaError_t launch_row_pipe<double>(bool, const RowArgs<double>&, int, size_t, cudaStream_t);
template cudaError_t row_pipe_blocks_per_sm<double>(bool, size_t, int*);
template cudaError_t launch_row_p2<double>(bool, const RowArgs<double>&, dim3, size_t, cudaStream_t);
template cudaError_t launch_zfused<double>(const ZfArgs<double>&, int, int, size_t, cudaStream_t);
template int zfused_max_clusters<double>(int, int, size_t);
template cudaError_t launch_zseq<double>(const ZseqArgs<double>&, int, int, size_t, cudaStream_t, int*);

}  // namespace sgs
