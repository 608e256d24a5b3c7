// Explicit instantiations of the tail factorization kernels (double, nb in [12, 16]).
#include "bm_tail_factor.cuh"

namespace bm {
namespace tail {
template void launch_tail_nb<double, 12>(const TailView<double> &, cudaStream_t, const TailSched *, cudaEvent_t *);
template void launch_tail_range<double, 12>(const TailView<double> &, cudaStream_t, const TailSched *, int, int,
                                             bool, cudaEvent_t *);
template cudaError_t prepare_nb<double, 12>();
template void launch_tail_nb<double, 16>(const TailView<double> &, cudaStream_t, const TailSched *, cudaEvent_t *);
template void launch_tail_range<double, 16>(const TailView<double> &, cudaStream_t, const TailSched *, int, int,
                                             bool, cudaEvent_t *);
template cudaError_t prepare_nb<double, 16>();
}  // namespace tail
}  // namespace bm
