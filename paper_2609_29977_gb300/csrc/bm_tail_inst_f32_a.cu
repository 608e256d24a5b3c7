// Explicit instantiations of the tail factorization kernels (float, nb in [2, 3, 4, 6, 8]).
#include "bm_tail_factor.cuh"
#include "bm_tail_rows.cuh"

namespace bm {
namespace tail {
template void launch_tail_nb<float, 2>(const TailView<float> &, cudaStream_t, const TailSched *, cudaEvent_t *);
template cudaError_t prepare_nb<float, 2>();
template void launch_tail_nb<float, 3>(const TailView<float> &, cudaStream_t, const TailSched *, cudaEvent_t *);
template cudaError_t prepare_nb<float, 3>();
template void launch_tail_nb<float, 4>(const TailView<float> &, cudaStream_t, const TailSched *, cudaEvent_t *);
template cudaError_t prepare_nb<float, 4>();
template void launch_tail_nb<float, 6>(const TailView<float> &, cudaStream_t, const TailSched *, cudaEvent_t *);
template cudaError_t prepare_nb<float, 6>();
template void launch_tail_nb<float, 8>(const TailView<float> &, cudaStream_t, const TailSched *, cudaEvent_t *);
template cudaError_t prepare_nb<float, 8>();
}  // namespace tail
template void rows::launch_tail_rows<float, 2>(const TailView<float> &, cudaStream_t);
template cudaError_t rows::prepare_rows<float, 2>();
template void rows::launch_tail_rows<float, 3>(const TailView<float> &, cudaStream_t);
template cudaError_t rows::prepare_rows<float, 3>();
template void rows::launch_tail_rows<float, 4>(const TailView<float> &, cudaStream_t);
template cudaError_t rows::prepare_rows<float, 4>();
template void rows::launch_tail_rows<float, 6>(const TailView<float> &, cudaStream_t);
template cudaError_t rows::prepare_rows<float, 6>();
template void rows::launch_tail_rows<float, 8>(const TailView<float> &, cudaStream_t);
template cudaError_t rows::prepare_rows<float, 8>();
}  // namespace bm
