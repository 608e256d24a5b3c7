// Launches of the coupling-column refinement of the mixed-precision factor
// (device bodies and the method in bm_coupling.cuh). Four launches after the
// FP32 tail factor, each with one thread-block cluster per tail for the
// level walks:
//   k_cx_bwd (pass 0)  X0 = L^-T L^-1 C^T
//   k_cx_residual      P = C^T - K X0 (float-float, grid-stride over rows)
//   k_cx_fwd           L^-1 P
//   k_cx_bwd (pass 1)  d = L^-T (...), X = X0 + d, U_i from X0 + d
// When the refinement is conditional (the handle's automatic mode), each
// kernel first reads the engage word that the root probe wrote and returns
// at once if it is clear.
#include "bm_coupling.cuh"

namespace bm {
namespace {
using namespace cx;

template <int NB>
__global__ void __launch_bounds__(XCfg<NB>::THREADS, XCfg<NB>::MINB) k_cx_bwd(CxView v, int pass, int CS, int *mark) {
  __shared__ __align__(16) float scr[XCfg<NB>::TEAMS * XCfg<NB>::SCR];
  pdl_wait();
  if (engaged(v)) {
    if (mark && pass == 0 && blockIdx.x == 0 && threadIdx.x == 0) *mark = 1;
    bwd_multi<NB>(v, blockIdx.x / CS, (int)mx::cluster_rank(), CS, pass, scr);
  }
  pdl_trigger();
}

template <int NB>
__global__ void __launch_bounds__(XCfg<NB>::THREADS, XCfg<NB>::MINB) k_cx_fwd(CxView v, int CS) {
  __shared__ __align__(16) float scr[XCfg<NB>::TEAMS * XCfg<NB>::SCR];
  pdl_wait();
  if (engaged(v)) fwd_multi<NB>(v, blockIdx.x / CS, (int)mx::cluster_rank(), CS, scr);
  pdl_trigger();
}

template <int NB>
__global__ void __launch_bounds__(256, 4) k_cx_residual(CxView v) {
  pdl_wait();
  if (engaged(v)) {
    const long nrow = (long)v.S * v.N * NB;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < nrow; e += (long)gridDim.x * blockDim.x) {
      const long br = e / NB;
      const int i = (int)(e - br * NB);
      const int s = (int)(br / v.N), k = (int)(br - (long)s * v.N);
      residual_row_multi<NB>(v, s, k, i);
    }
  }
  pdl_trigger();
}

int pick_cluster_cx(int S) {
  int cs = 1;
  while (cs < 8 && S * cs * 2 <= 152) cs <<= 1;
  return cs;
}

template <typename... KArgs, typename... Args>
cudaError_t launch_cx_shape(void (*kern)(KArgs...), unsigned grid, unsigned block, size_t smem, int CS,
                            cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  attr[1].id = cudaLaunchAttributeClusterDimension;
  attr[1].val.clusterDim.x = CS;
  attr[1].val.clusterDim.y = 1;
  attr[1].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = CS > 1 ? 2 : 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

template <typename... KArgs, typename... Args>
cudaError_t launch_cx(void (*kern)(KArgs...), unsigned grid, unsigned block, int CS, cudaStream_t st,
                      Args... args) {
  return launch_cx_shape(kern, grid, block, 0, CS, st, args...);
}

template <int NB>
void launch_nb(const CxView &v, int *mark, cudaStream_t st) {
  const int CS = pick_cluster_cx(v.S);
  const unsigned grid = (unsigned)(v.S * CS);
  constexpr unsigned THR = XCfg<NB>::THREADS;
  launch_cx(k_cx_bwd<NB>, grid, THR, CS, st, v, 0, CS, mark);
  const long rows = (long)v.S * v.N * NB;
  long blocks = (rows + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  launch_cx(k_cx_residual<NB>, (unsigned)blocks, 256u, 1, st, v);
  launch_cx(k_cx_fwd<NB>, grid, THR, CS, st, v, CS);
  launch_cx(k_cx_bwd<NB>, grid, THR, CS, st, v, 1, CS, (int *)nullptr);
}

}  // namespace

// Refines the coupling columns of a factored FP32 tail set (v.U receives the
// FP64 local Schur updates). mark, if not null, is set to 1 by the first
// kernel when the refinement runs.
void coupling_launch(const CxView &v, int nb, int *mark, cudaStream_t st) {
  switch (nb) {
#define X(n)                          \
  case n:                             \
    launch_nb<n>(v, mark, st); \
    break;
    BM_TAIL_NB_LIST(X)
#undef X
  }
}

}  // namespace bm
