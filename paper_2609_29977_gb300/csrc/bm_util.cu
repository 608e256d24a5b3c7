// Small utilities exposed through the C ABI.
#include "bm_team.cuh"

namespace {

__global__ void k_round_fp32(const double *__restrict__ src, float *__restrict__ dst, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = bm::d2f_rn(src[i]);
}

}  // namespace

extern "C" bm_status bm_round_to_fp32(const double *src, float *dst, size_t n, void *stream) {
  if ((!src || !dst) && n) return BM_ERR_INVALID_ARG;
  if (n == 0) return BM_OK;
  size_t blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_round_fp32<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(src, dst, n);
  return cudaGetLastError() == cudaSuccess ? BM_OK : BM_ERR_CUDA;
}
