// Internal definitions shared by the CUDA translation units of the library.
//
// Indexing of the tail permutation (Sec. IV-A). A tail of N stages is read as
// a chain of positions p = 1..N with p = N + 1 - k for natural 1-based stage
// k: Omega_i reverses the stages, positions 1..N-1 carry (x_N, ..., x_2), on
// which Gamma_{N-1} acts, and position N is x_1, kept last. Gamma_{N-1}
// (Sec. II) eliminates first every other position starting with the first
// (the odd ones), then recurses on the rest, so position p belongs to level
// ctz(p) and the chain has Lc = bit_length(N-1) levels. At level l the chain
// still holds the multiples of 2^l and x_1; the eliminated position p (an
// odd multiple of 2^l) has the left neighbour p - 2^l (when p > 2^l) and
// the right neighbour p + 2^l, or x_1 when p + 2^l > N - 1. Blocks of one
// level are never neighbours, so they are eliminated concurrently.
//
// Every per-stage array of the library is stored by NATURAL stage index
// k - 1 = N - p, so exported factors line up with the input blocks.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/bm.h"

namespace bm {

__host__ __device__ inline int ctz32(int p) {
#ifdef __CUDA_ARCH__
  return __ffs(p) - 1;
#else
  return __builtin_ctz((unsigned)p);
#endif
}

// Number of odd-even levels of the N-1 chain positions.
__host__ __device__ inline int chain_levels(int N) {
  int n = N - 1, l = 0;
  while (n > 0) { ++l; n >>= 1; }
  return l;
}

// Tasks of factor/forward launch l: l = 0 -> the odd positions; l >= 1 ->
// every remaining position (multiples of 2^l) plus x_1.
__host__ __device__ inline int level_tasks(int N, int l) {
  return l == 0 ? N / 2 : ((N - 1) >> l) + 1;
}
__device__ inline int level_task_pos(int N, int l, int j) {
  if (l == 0) return 2 * j + 1;
  int cnt = (N - 1) >> l;
  return j < cnt ? (j + 1) << l : N;
}
// Positions eliminated at level l (odd multiples of 2^l that are <= N-1).
__host__ __device__ inline int level_elims(int N, int l) {
  return (((N - 1) >> l) + 1) / 2;
}

// Device status word (sticky until the next bm_factor).
struct Status {
  int code;       // bm_status
  int scenario;   // 0-based, -1 root
  int stage;      // 1-based natural stage, 0 root
  int iters;      // refinement steps
  double eta;     // refinement: componentwise backward error of the iterate
};

__device__ inline void report_not_spd(Status *st, int scenario, int stage) {
  if (atomicCAS(&st->code, 0, (int)BM_ERR_NOT_SPD) == 0) {
    st->scenario = scenario;
    st->stage = stage;
  }
}

// Root reduction of Alg. 1 step 4 for one entry (i, j): sum_s U_s[i][j] in
// the library's fixed order -- four accumulators over s = k mod 4, each in
// increasing s, combined as (a0 + a1) + (a2 + a3) -- so that every code path
// (single system, batch) gets the same bits for the same system.
__device__ inline double root_sum(const double *U, int S, int nr, int i, int j) {
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  const size_t stride = (size_t)nr * nr, off = (size_t)i * nr + j;
  int s = 0;
  // sixteen loads in flight per step; accumulator k still adds U[s + k],
  // U[s + 4 + k], ... in increasing s, so the bits do not depend on the unroll
  for (; s + 16 <= S; s += 16) {
    double v[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __ldcg(U + (size_t)(s + k) * stride + off);
#pragma unroll
    for (int k = 0; k < 16; ++k) a[k & 3] += v[k];
  }
  for (; s + 4 <= S; s += 4) {
#pragma unroll
    for (int k = 0; k < 4; ++k) a[k] += __ldcg(U + (size_t)(s + k) * stride + off);
  }
  for (int k = 0; s < S; ++s, ++k) a[k] += __ldcg(U + (size_t)s * stride + off);
  return (a[0] + a[1]) + (a[2] + a[3]);
}

// Views passed to the FP64 kernels (by value).
struct F64View {
  int S, N, nb, nr, Lc;
  const double *D, *E, *C, *R;
  double *Ld, *Ll, *Lr;   // [S][N][nb*nb]
  double *Dt, *W;         // [S][N][nb*nb] level workspace (updated diagonals, fill couplings)
  double *F, *U;          // [S][nr*nb], [S][nr*nr]
  double *LR, *Rt;        // [nr*nr]
  double *invd;           // [S][N][nb] inverse diagonals 1/(L_pp)_jj of the tail factor
  double *y, *zt;         // [S][N][nb] solve workspace
  double *tb;             // [S][nr]
  unsigned *tickets;      // last-block counters
  Status *status;
};

// View of one system's tail factor for the templated tail kernels
// (T = double on the FP64 path, float for the tails of the mixed path). The
// inputs are always FP64; the coupling factor F and local updates U are
// always FP64.
template <typename T>
struct TailView {
  int S, N, nb, nr, Lc;
  const double *D, *E, *C, *R;
  T *Ld, *Ll, *Lr;   // [S][N][nb*nb]
  T *Dt, *W;         // [S][N][nb*nb] level workspace
  T *invd;           // [S][N][nb]
  double *F, *U;     // [S][nr*nb], [S][nr*nr]
  Status *status;
};

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Block sizes with compile-time tail kernels.
#define BM_TAIL_NB_LIST(X) X(2) X(3) X(4) X(6) X(8) X(12) X(16) X(24) X(32) X(48)
// Block sizes whose FP32 tails use the register-row kernels (bm_tail_rows.cuh).
#define BM_ROWS_NB_LIST(X) X(2) X(3) X(4) X(6) X(8) X(12) X(16) X(24) X(32)

// First level handled by the per-tail top kernel: the first one with at
// most four positions per tail (Lc when none).
inline int top_level(int N) {
  const int Lc = chain_levels(N);
  for (int l = 0; l < Lc; ++l) {
    const int tasks = l == 0 ? N / 2 : ((N - 1) >> l) + 1;
    if (tasks <= 4) return l;
  }
  return Lc;
}

bool tail_nb_supported(int nb);
cudaError_t tail_factor_prepare();
template <typename T>
void tail_factor_launch(const TailView<T> &v, cudaStream_t st);

// Launch with programmatic stream serialization (PDL): the kernel may begin
// while its predecessor drains and waits in griddepcontrol.wait.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

}  // namespace bm
