// Explicit instantiations of the tail factorization kernels (float, nb in [12, 16]).
#include "bm_tail_factor.cuh"

namespace bm {
namespace tail {
template void launch_tail_nb<float, 12>(const TailView<float> &, cudaStream_t);
template cudaError_t prepare_nb<float, 12>();
template void launch_tail_nb<float, 16>(const TailView<float> &, cudaStream_t);
template cudaError_t prepare_nb<float, 16>();
}  // namespace tail
}  // namespace bm
