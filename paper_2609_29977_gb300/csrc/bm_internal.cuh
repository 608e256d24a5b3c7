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
  int coupled;    // mixed precision: the coupling columns were refined in the last factor
  unsigned spread; // mixed precision: max over tails of (max/min FP32 pivot)^2, float bits
  int ffbad;      // mixed precision: an entry of K or x is outside the float-float residual's range
  double eta;     // refinement: componentwise backward error of the iterate
};

__device__ inline void report_not_spd(Status *st, int scenario, int stage) {
  if (atomicCAS(&st->code, 0, (int)BM_ERR_NOT_SPD) == 0) {
    st->scenario = scenario;
    st->stage = stage;
  }
}

// Root reduction of Alg. 1 step 4 for one entry (i, j): sum_s U_s[i][j] in
// the library's fixed order. Lane l of a warp adds U_l, U_{l+32}, ... in
// increasing s; the 32 partial sums p_l are then combined by the butterfly
// p_l <- p_l + p_{l xor o} for o = 16, 8, 4, 2, 1 (addition commutes
// exactly, so every lane ends with the same bits). Every code path (single
// system, batch, serving) uses this order, so a system's root gets the same
// bits wherever it is factored. Call with all 32 lanes of a warp.
__device__ inline double root_sum_warp(const double *U, int S, int nr, int i, int j) {
  const int lane = threadIdx.x & 31;
  const size_t stride = (size_t)nr * nr, off = (size_t)i * nr + j;
  double acc = 0.0;
  int s = lane;
  // four loads in flight per lane; each lane still adds in increasing s
  for (; s + 96 < S; s += 128) {
    const double a = __ldcg(U + (size_t)s * stride + off), b = __ldcg(U + (size_t)(s + 32) * stride + off);
    const double c = __ldcg(U + (size_t)(s + 64) * stride + off), d = __ldcg(U + (size_t)(s + 96) * stride + off);
    acc += a;
    acc += b;
    acc += c;
    acc += d;
  }
  for (; s < S; s += 32) acc += __ldcg(U + (size_t)s * stride + off);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  return acc;
}

// The same order evaluated by one thread.
__device__ inline double root_sum_serial(const double *U, int S, int nr, int i, int j) {
  const size_t stride = (size_t)nr * nr, off = (size_t)i * nr + j;
  double p[32];
#pragma unroll
  for (int l = 0; l < 32; ++l) p[l] = 0.0;
  for (int s = 0; s < S; ++s) p[s & 31] += __ldcg(U + (size_t)s * stride + off);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    double q[32];
#pragma unroll
    for (int l = 0; l < 32; ++l) q[l] = p[l] + p[l ^ o];
#pragma unroll
    for (int l = 0; l < 32; ++l) p[l] = q[l];
  }
  return p[0];
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
  // FP64 path: the top kernel's last CTA also forms R~ (Rt) and L_R (LR)
  // when LR is set (ticket tickets[0]); null elsewhere
  double *Rt, *LR;
  unsigned *tickets;
  // index of this view's first tail among all tails of the system (a view
  // over a range of tails reports failures with system-wide indices)
  int s0;
};

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Launch schedule of the FP64 tail factor: the first level that the per-tail
// top kernel takes over (one CTA per tail), and the team size (lanes per
// chain position) of each grid-wide level launch before it.
struct TailSched {
  int top;
  int team[32];
};

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
// sc: schedule of the FP64 tail factor (null: the default rule); ev: if not
// null, top + 2 events recorded before the first launch and after each one.
template <typename T>
void tail_factor_launch(const TailView<T> &v, cudaStream_t st, const TailSched *sc = nullptr,
                        cudaEvent_t *ev = nullptr);
// The default schedule, and the autotuned one (times candidate team sizes
// per level and top levels on the given inputs, synchronizing st).
void tail_factor_launch_range(const TailView<double> &v, cudaStream_t st, const TailSched *sc, int lo, int hi,
                              bool top);
void tail_default_schedule(int S, int N, int nb, TailSched *sc);
bool tail_factor_tune(const TailView<double> &v, cudaStream_t st, TailSched *best);

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
