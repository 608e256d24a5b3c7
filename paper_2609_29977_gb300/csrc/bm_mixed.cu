// Mixed-precision path (FP32 tails, FP64 root and refinement): not built yet.
#include "bm_internal.cuh"

namespace bm {
struct MixedState {};
size_t mixed_bytes(int, int, int, int) { return 0; }
cudaError_t mixed_prepare(int, int) { return cudaErrorNotSupported; }
MixedState *mixed_create(int, int, int, int, void *, size_t, Status *, unsigned *) { return nullptr; }
void mixed_destroy(MixedState *) {}
void mixed_launch_factor(MixedState *, const double *, const double *, const double *, const double *,
                         cudaStream_t) {}
void mixed_launch_solve(MixedState *, const double *, double *, int, double, cudaStream_t) {}
void mixed_launch_export(MixedState *, double *, double *, double *, double *, double *, cudaStream_t) {}
}  // namespace bm
