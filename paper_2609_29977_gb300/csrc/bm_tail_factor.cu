// Dispatch of the tail factorization on the block size (Alg. 1, steps 1-3).
// The kernels are defined in bm_tail_factor.cuh and instantiated in
// bm_tail_inst_*.cu.
#include <mutex>

#include "bm_tail_factor.cuh"
#include "bm_tail_rows.cuh"

namespace bm {
namespace tail {
#define X(n)                                                                         \
  extern template void launch_tail_nb<double, n>(const TailView<double> &, cudaStream_t); \
  extern template void launch_tail_nb<float, n>(const TailView<float> &, cudaStream_t);   \
  extern template cudaError_t prepare_nb<double, n>();                              \
  extern template cudaError_t prepare_nb<float, n>();
BM_TAIL_NB_LIST(X)
#undef X
}  // namespace tail
namespace rows {
#define X(n)                                                                                  \
  extern template void launch_tail_rows<float, n>(const TailView<float> &, cudaStream_t); \
  extern template cudaError_t prepare_rows<float, n>();
BM_ROWS_NB_LIST(X)
#undef X
extern template void launch_tail_rows_w<float, 48>(const TailView<float> &, cudaStream_t);
extern template cudaError_t prepare_rows_w<float, 48>();
}  // namespace rows

bool tail_nb_supported(int nb) {
  switch (nb) {
#define X(n) case n:
    BM_TAIL_NB_LIST(X)
#undef X
    return true;
  }
  return false;
}

cudaError_t tail_factor_prepare() {
  static std::mutex mu;
  static bool done[64] = {false};
  std::lock_guard<std::mutex> lock(mu);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return cudaErrorUnknown;
  if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
  cudaError_t e = cudaSuccess;
#define X(n)                                                   \
  if (e == cudaSuccess) e = tail::prepare_nb<double, n>();     \
  if (e == cudaSuccess) e = tail::prepare_nb<float, n>();
  BM_TAIL_NB_LIST(X)
#undef X
#define X(n) \
  if (e == cudaSuccess) e = rows::prepare_rows<float, n>();
  BM_ROWS_NB_LIST(X)
#undef X
  if (e == cudaSuccess) e = rows::prepare_rows_w<float, 48>();
  if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
  return e;
}

// Tail levels and x_1 of the factor (the root step is launched separately).
// FP32 tails use the register-row kernels (two-warp teams for nb = 48).
template <typename T>
void tail_factor_launch(const TailView<T> &v, cudaStream_t st) {
  if (sizeof(T) == 4) {
    switch (v.nb) {
#define X(n)                                                                        \
  case n:                                                                           \
    rows::launch_tail_rows<float, n>(*reinterpret_cast<const TailView<float> *>(&v), st); \
    return;
      BM_ROWS_NB_LIST(X)
#undef X
      case 48:
        rows::launch_tail_rows_w<float, 48>(*reinterpret_cast<const TailView<float> *>(&v), st);
        return;
    }
  }
  switch (v.nb) {
#define X(n)                           \
  case n:                              \
    tail::launch_tail_nb<T, n>(v, st); \
    break;
    BM_TAIL_NB_LIST(X)
#undef X
  }
}
template void tail_factor_launch<double>(const TailView<double> &, cudaStream_t);
template void tail_factor_launch<float>(const TailView<float> &, cudaStream_t);

}  // namespace bm
