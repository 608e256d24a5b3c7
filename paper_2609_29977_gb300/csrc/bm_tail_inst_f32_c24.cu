// Explicit instantiations of the tail factorization kernels (float, nb = 24).
#include "bm_tail_factor.cuh"
#include "bm_tail_rows.cuh"

namespace bm {
namespace tail {
template void launch_tail_nb<float, 24>(const TailView<float> &, cudaStream_t, const TailSched *, cudaEvent_t *);
template cudaError_t prepare_nb<float, 24>();
}  // namespace tail
template void rows::launch_tail_rows<float, 24>(const TailView<float> &, cudaStream_t);
template cudaError_t rows::prepare_rows<float, 24>();
}  // namespace bm
