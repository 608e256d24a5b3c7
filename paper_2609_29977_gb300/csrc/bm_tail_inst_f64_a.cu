// Explicit instantiations of the tail factorization kernels (double, nb in [2, 3, 4, 6, 8]).
#include "bm_tail_factor.cuh"

namespace bm {
namespace tail {
template void launch_tail_nb<double, 2>(const TailView<double> &, cudaStream_t, const TailSched *, cudaEvent_t *);
template void launch_tail_range<double, 2>(const TailView<double> &, cudaStream_t, const TailSched *, int, int,
                                             bool, cudaEvent_t *);
template cudaError_t prepare_nb<double, 2>();
template void launch_tail_nb<double, 3>(const TailView<double> &, cudaStream_t, const TailSched *, cudaEvent_t *);
template void launch_tail_range<double, 3>(const TailView<double> &, cudaStream_t, const TailSched *, int, int,
                                             bool, cudaEvent_t *);
template cudaError_t prepare_nb<double, 3>();
template void launch_tail_nb<double, 4>(const TailView<double> &, cudaStream_t, const TailSched *, cudaEvent_t *);
template void launch_tail_range<double, 4>(const TailView<double> &, cudaStream_t, const TailSched *, int, int,
                                             bool, cudaEvent_t *);
template cudaError_t prepare_nb<double, 4>();
template void launch_tail_nb<double, 6>(const TailView<double> &, cudaStream_t, const TailSched *, cudaEvent_t *);
template void launch_tail_range<double, 6>(const TailView<double> &, cudaStream_t, const TailSched *, int, int,
                                             bool, cudaEvent_t *);
template cudaError_t prepare_nb<double, 6>();
template void launch_tail_nb<double, 8>(const TailView<double> &, cudaStream_t, const TailSched *, cudaEvent_t *);
template void launch_tail_range<double, 8>(const TailView<double> &, cudaStream_t, const TailSched *, int, int,
                                             bool, cudaEvent_t *);
template cudaError_t prepare_nb<double, 8>();
}  // namespace tail
}  // namespace bm
