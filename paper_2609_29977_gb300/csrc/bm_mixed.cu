// Mixed-precision path (BM_PREC_FP32_IR): FP32 tails, FP64 root, FP64
// iterative refinement on the full system. Not in the paper; its steps are
// the paper's (Alg. 1 for the factor, Alg. 2 for each correction solve) with
// the tail blocks held in FP32.
//
// Factor: the tail factor of Alg. 1 steps 1-3 in FP32 (bm_tail_factor.cuh,
// T = float); F_{i,1} and U_i = F_{i,1} F_{i,1}^T in FP64 from the FP32
// L_{i,1}; the root reduction R - sum U_i and L_R = chol in FP64.
//
// Solve: x_0 = 0, rho_0 = r; for k = 0..max_refine:
//   d = M^{-1} rho_k  (Alg. 2 with FP32 tails and an FP64 root step),
//   x += d (FP64), rho_{k+1} = r - K x (FP64, from the caller's D, E, C, R),
//   stop when the componentwise backward error
//   omega = max_i |rho_i| / (|K| |x| + |r|)_i <= tol (Oettli-Prager), or
//   when omega fails to halve from one iteration to the next.
// Each iteration is three launches: forward tail substitution whose last CTA
// does the root step, backward tail substitution fused with x += d, and the
// residual whose last CTA applies the stopping test.
//  * In a captured graph the iterations are the body of one conditional
//    WHILE node: the forward kernel first sets the loop condition to 0, and
//    the residual's last CTA sets it back to 1 only when another iteration
//    is to run, so the loop ends on the device after the last useful
//    iteration (at most max_refine + 1 bodies) with no host round trip.
//  * Launched directly, the max_refine + 1 iterations are unrolled; once the
//    stopping test holds it raises a device flag, and every later launch
//    checks the flag first and returns.
// Both forms run the same kernels on the same data: the results are
// bitwise identical.
#include <cuda_runtime.h>

#include <mutex>
#include <new>

#include "bm_coupling.cuh"
#include "bm_mixed.cuh"

namespace bm {
namespace {
using namespace mx;

// CTAs of the residual and root-term launches (grid-stride over the rows of
// the tails, at least one CTA per root row): also the number of root-term
// parts the forward kernel sums. At most max(152 * 8, nr).
__host__ __device__ inline int xt_blocks(int S, int N, int nb, int nr) {
  const long rows = (long)S * N * nb;
  long blocks = (rows + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks < nr) blocks = nr;
  return (int)blocks;
}

// iter >= 0: a directly launched iteration; iter < 0: the body of a graph
// loop, whose iteration index is read from the control block and whose
// condition handle is cond.
template <int NB>
__global__ void __launch_bounds__(256) k_mixed_fwd(MixedState m, const double *__restrict__ r, double *x, int iter,
                                                    int CS, cudaGraphConditionalHandle cond) {
  __shared__ float sY[MCfg<NB>::TEAMS][NB];
  __shared__ double sR[64 * 64 + 64 + 64];
  pdl_wait();
  // the loop stops after this iteration unless its stopping test says otherwise
  if (iter < 0 && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, 0u);
  if (ir_done(m.ctl)) return;
  const int it = ir_iter(m.ctl, iter);
  const double *rhs = it == 0 ? r : m.rho;
  fwd_tail<NB>(m, rhs, blockIdx.x / CS, (int)cluster_rank(), CS, sY);
  if (last_cta(&m.tickets[2], gridDim.x)) root_step<NB>(m, rhs, x, it, sR, coupled(m) ? xt_blocks(m.S, m.N, NB, m.nr) : m.S);
}

template <int NB>
__global__ void __launch_bounds__(256) k_mixed_bwd(MixedState m, double *x, int iter, int CS) {
  __shared__ float sX[MCfg<NB>::TEAMS][NB];
  pdl_wait();
  if (ir_done(m.ctl)) return;
  bwd_tail<NB>(m, x, ir_iter(m.ctl, iter), blockIdx.x / CS, (int)cluster_rank(), CS, sX);
}

// rho = r - K x in FP64 and the componentwise backward error of the
// iterate; one thread per row of the tails (grid-stride; every lane of an
// FP64 warp instruction does useful work), one more CTA-strided pass over
// the root rows. With refined coupling columns each CTA then leaves its part
// of the next correction's root term X^T rho in tb. The last CTA applies
// the stopping test.
template <int NB>
__global__ void __launch_bounds__(256, 5) k_mixed_residual(MixedState m, const double *__restrict__ r,
                                                         const double *__restrict__ x, int iter, int max_iter,
                                                         double tol, cudaGraphConditionalHandle cond) {
  __shared__ unsigned sroot;
  pdl_wait();
  if (ir_done(m.ctl)) return;
  const int it = ir_iter(m.ctl, iter);
  const long nrow = (long)m.S * m.N * NB;
  // float-float unless the handle computes FP64 residuals or an entry of K
  // or x left the float-float range (uniform over the grid)
  const bool ffr = m.ffres && __ldcg(&m.status->ffbad) == 0;
  float om = 0.0f;
  if (ffr) {
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < nrow; e += (long)gridDim.x * blockDim.x) {
      const long br = e / NB;
      const int i = (int)(e - br * NB);
      const int s = (int)(br / m.N), k = (int)(br - (long)s * m.N);
      om = fmaxf(om, residual_row_ff<NB>(m, r, x, s, k, i));
    }
  } else {
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < nrow; e += (long)gridDim.x * blockDim.x) {
      const long br = e / NB;
      const int i = (int)(e - br * NB);
      const int s = (int)(br / m.N), k = (int)(br - (long)s * m.N);
      om = fmaxf(om, residual_row<NB>(m, r, x, s, k, i));
    }
  }
  omega_publish(m.ctl, om);
  // each thread reads back only the rho rows it wrote
  if (coupled(m)) xt_grid(m, m.rho, NB);
  // root rows; their omega goes through the same maximum
  if (threadIdx.x == 0) sroot = 0u;
  __syncthreads();
  for (int c = blockIdx.x; c < m.nr; c += gridDim.x) {
    const float oc = residual_root_row(m, r, x, NB, c);
    if (threadIdx.x == 0) sroot = max(sroot, __float_as_uint(oc));
  }
  __syncthreads();
  if (threadIdx.x == 0 && sroot) atomicMax(&m.ctl->wmax, sroot);
  if (last_cta(&m.tickets[3], gridDim.x) && threadIdx.x == 0) {
    const bool more = ir_stop(m, 0.0f, it, max_iter, ffr ? tol - kFFBeta : tol);
    if (iter < 0 && more) cudaGraphSetConditional(cond, 1u);
  }
}

// Root terms of the first correction with refined coupling columns: the
// per-CTA parts of X^T r over the same grid-stride walk as the residual
// kernel (which leaves those of the later corrections). Returns at once
// without refined columns.
template <int NB>
__global__ void __launch_bounds__(256) k_mixed_xt(MixedState m, const double *__restrict__ r) {
  pdl_wait();
  if (coupled(m)) xt_grid(m, r, NB);
}

// Pivot spread of the FP32 tail factor for the automatic mode's probe:
// (max_j L_jj / min_j L_jj)^2 over the pivots of tail blockIdx.x (from the
// inverse pivots invd), folded into the status word's maximum.
__global__ void __launch_bounds__(256) k_pivot_spread(const float *__restrict__ invd, int N, int nb, Status *st) {
  __shared__ float smax[8], smin[8];
  pdl_wait();
  const int rows = N * nb;
  const float *p = invd + (size_t)blockIdx.x * rows;
  float mx = 0.0f, mn = __int_as_float(0x7f800000);
  for (int e = threadIdx.x; e < rows; e += blockDim.x) {
    const float v = fabsf(p[e]);
    mx = fmaxf(mx, v);
    mn = fminf(mn, v);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
  }
  if ((threadIdx.x & 31) == 0) {
    smax[threadIdx.x >> 5] = mx;
    smin[threadIdx.x >> 5] = mn;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      mx = fmaxf(mx, smax[w]);
      mn = fminf(mn, smin[w]);
    }
    mx = fmaxf(mx, smax[0]);
    mn = fminf(mn, smin[0]);
    const float ratio = mn > 0.0f ? (mx / mn) * (mx / mn) : __int_as_float(0x7f7fffff);
    atomicMax(&st->spread, __float_as_uint(fminf(ratio, __int_as_float(0x7f7fffff))));
  }
  pdl_trigger();
}

// Widen the FP32 tail factor for export.
__global__ void k_widen(const float *__restrict__ src, double *__restrict__ dst, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = f2d_exact(src[i]);
}

// K split into hi + lo floats for the float-float residual: D as full
// symmetric rows (its lower triangle mirrored), E as stored. Sets
// status->ffbad if a nonzero entry is outside the float-float range. D is
// staged a few blocks at a time in shared memory (read and written
// contiguously; the mirror is read from shared memory), E streams.
template <int NB>
struct SplitCfg {
  static constexpr int NB2 = NB * NB;
  static constexpr int BPI = NB2 >= 2048 ? 1 : 2048 / NB2;   // D blocks per staging round
};

template <int NB>
__global__ void __launch_bounds__(256) k_ff_split(MixedState m) {
  constexpr int NB2 = NB * NB, BPI = SplitCfg<NB>::BPI;
  __shared__ double sD[BPI * NB2];
  pdl_wait();
  bool bad = false;
  const long nblk = (long)m.S * m.N;
  for (long b0 = (long)blockIdx.x * BPI; b0 < nblk; b0 += (long)gridDim.x * BPI) {
    const int nb = nblk - b0 < BPI ? (int)(nblk - b0) : BPI;
    const double *src = m.D + b0 * NB2;
    __syncthreads();
    for (int e = threadIdx.x; e < nb * NB2; e += blockDim.x) sD[e] = src[e];
    __syncthreads();
    for (int e = threadIdx.x; e < nb * NB2; e += blockDim.x) {
      const int blk = e / NB2, w = e - blk * NB2, i = w / NB, j = w - i * NB;
      const double v = j <= i ? sD[e] : sD[blk * NB2 + j * NB + i];
      float h, l;
      ff::split_d(v, h, l);
      m.Kdh[b0 * NB2 + e] = h;
      m.Kdl[b0 * NB2 + e] = l;
      bad |= ff::out_of_range(v);
    }
  }
  const long ne = (long)m.S * (m.N - 1) * NB2;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += (long)gridDim.x * blockDim.x) {
    const double v = m.E[e];
    float h, l;
    ff::split_d(v, h, l);
    m.Keh[e] = h;
    m.Kel[e] = l;
    bad |= ff::out_of_range(v);
  }
  if (bad) m.status->ffbad = 1;
  pdl_trigger();
}

// x split into hi + lo floats (bm_residual; the refinement splits its
// iterate in the backward kernel).
__global__ void __launch_bounds__(256) k_x_split(MixedState m, const double *__restrict__ x) {
  const long n = (long)m.S * m.N * m.nb;
  bool bad = false;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    const double v = x[e];
    ff::split_d(v, m.xh[e], m.xl[e]);
    bad |= ff::out_of_range(v);
  }
  if (bad) m.status->ffbad = 1;
}

// rho = r - K x with the refinement's arithmetic (bm_residual): m.rho is
// the caller's array.
template <int NB>
__global__ void __launch_bounds__(256) k_residual_out(MixedState m, const double *__restrict__ r,
                                                       const double *__restrict__ x) {
  const long nrow = (long)m.S * m.N * NB;
  const bool ffr = m.ffres && __ldcg(&m.status->ffbad) == 0;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < nrow; e += (long)gridDim.x * blockDim.x) {
    const long br = e / NB;
    const int i = (int)(e - br * NB);
    const int s = (int)(br / m.N), k = (int)(br - (long)s * m.N);
    if (ffr)
      residual_row_ff<NB>(m, r, x, s, k, i);
    else
      residual_row<NB>(m, r, x, s, k, i);
  }
  for (int c = blockIdx.x; c < m.nr; c += gridDim.x) residual_root_row(m, r, x, NB, c);
}

// Automatic mode (cmode 1): a refinement that ended BM_ERR_NOT_CONVERGED
// while the factor's probe had kept the FP32-based root is resumed with
// refined coupling columns. This kernel decides (one thread): it clears the
// failure, marks the columns refined for this factor, restarts the
// iteration count at 1 (the next correction starts from the last residual)
// and, inside a captured graph, sets the condition of the conditional node
// that holds the resumed refinement.
__global__ void k_retry_arm(MixedState m, int max_iter, cudaGraphConditionalHandle cond, int graph) {
  pdl_wait();
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    IRCtl *c = m.ctl;
    Status *st = m.status;
    const bool arm = m.cmode == 1 && max_iter >= 1 && st->code == (int)BM_ERR_NOT_CONVERGED && st->coupled == 0;
    if (arm) {
      c->retry = 1;
      st->coupled = 1;
      st->code = 0;
      c->converged = 0;
      c->wmax = 0u;
      c->loop = 1;
      c->omega_prev = __longlong_as_double(0x7ff0000000000000ll);
    }
    if (graph) cudaGraphSetConditional(cond, arm ? 1u : 0u);
  }
  pdl_trigger();
}

// Root terms X^T rho of the resumed refinement's first correction (the
// residual kernel left none: the columns were not refined then).
template <int NB>
__global__ void __launch_bounds__(256) k_retry_xt(MixedState m) {
  pdl_wait();
  if (*((volatile const int *)&m.ctl->retry)) xt_grid(m, m.rho, NB);
  pdl_trigger();
}

int pick_cluster(int S) {
  int cs = 1;
  while (cs < 8 && S * cs * 2 <= 152) cs <<= 1;
  return cs;
}

// pdl: allow programmatic dependent launch after the previous kernel.
template <typename... KArgs, typename... Args>
void launch_cluster(void (*kern)(KArgs...), unsigned grid, unsigned block, int CS, bool pdl, cudaStream_t st,
                    Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = pdl ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  cudaLaunchKernelEx(&cfg, kern, args...);
}

template <typename... KArgs, typename... Args>
void launch_plain(void (*kern)(KArgs...), unsigned grid, unsigned block, size_t smem, bool pdl, cudaStream_t st,
                  Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = pdl ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kern, args...);
}

// One iteration (iter >= 0), or the body of the graph loop (iter = -1).
template <int NB>
void launch_iteration(const MixedState &m, const double *r, double *x, int iter, int max_iter, double tol,
                      cudaStream_t st, cudaGraphConditionalHandle cond, bool pdl) {
  const int CS = pick_cluster(m.S);
  const unsigned grid = (unsigned)(m.S * CS);
  launch_cluster(k_mixed_fwd<NB>, grid, 256, CS, pdl, st, m, r, x, iter, CS, cond);
  launch_cluster(k_mixed_bwd<NB>, grid, 256, CS, pdl, st, m, x, iter, CS);
  const int blocks = xt_blocks(m.S, m.N, NB, m.nr);
  launch_plain(k_mixed_residual<NB>, (unsigned)blocks, 256, 0, pdl, st, m, r, (const double *)x, iter, max_iter, tol,
               cond);
}

// Adds the refinement loop to the graph being captured on st: a conditional
// WHILE node (condition 1 at every graph launch) after st's current
// dependencies, whose body graph is captured from body_st (with programmatic
// launches between its kernels when body_pdl is set).
template <int NB>
cudaError_t capture_loop(const MixedState &m, const double *r, double *x, int max_iter, double tol,
                         cudaStream_t st, cudaStream_t body_st, bool body_pdl) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t *deps = nullptr;
  const cudaGraphEdgeData *edges = nullptr;
  size_t ndeps = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, &edges, &ndeps);
  if (e != cudaSuccess) return e;
  if (cs != cudaStreamCaptureStatusActive || !g) return cudaErrorStreamCaptureInvalidated;
  cudaGraphConditionalHandle cond = 0;
  e = cudaGraphConditionalHandleCreate(&cond, g, 1u, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) return e;
  cudaGraphNodeParams p = {};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = cond;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  e = cudaGraphAddNode(&node, g, deps, edges, ndeps, &p);
  if (e != cudaSuccess) return e;
  cudaGraph_t body = p.conditional.phGraph_out[0];
  e = cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
  if (e != cudaSuccess) return e;
  e = cudaStreamBeginCaptureToGraph(body_st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  launch_iteration<NB>(m, r, x, -1, max_iter, tol, body_st, cond, body_pdl);
  const cudaError_t el = cudaPeekAtLastError();
  cudaGraph_t out = nullptr;
  e = cudaStreamEndCapture(body_st, &out);
  return el != cudaSuccess ? el : e;
}

// The resumed refinement's launches after the arm kernel: coupling-column
// refinement and root (both gated by ctl->retry), root terms, then the
// iterations (a loop node when body_st is set, else max_iter unrolled
// iterations that return at once unless armed).
void coupling_launch_cx(const MixedState &m, int *on, cudaStream_t st);
void retry_root(const MixedState &m, cudaStream_t st);

template <int NB>
cudaError_t launch_retry_body(const MixedState &m, const double *r, double *x, int max_iter, double tol,
                              cudaStream_t st, cudaStream_t body_st, bool pdl) {
  coupling_launch_cx(m, &m.ctl->retry, st);
  retry_root(m, st);
  launch_plain(k_retry_xt<NB>, (unsigned)xt_blocks(m.S, m.N, NB, m.nr), 256, 0, true, st, m);
  if (body_st) return capture_loop<NB>(m, r, x, max_iter, tol, st, body_st, pdl);
  for (int it = 1; it <= max_iter; ++it) launch_iteration<NB>(m, r, x, it, max_iter, tol, st, 0, true);
  return cudaPeekAtLastError();
}

// Captured form: the arm kernel, then a conditional IF node whose body
// (captured from if_st, its loop body from body_st) is launch_retry_body.
template <int NB>
cudaError_t capture_retry(const MixedState &m, const double *r, double *x, int max_iter, double tol,
                          cudaStream_t st, cudaStream_t if_st, cudaStream_t body_st, bool pdl) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, nullptr, nullptr, nullptr);
  if (e != cudaSuccess) return e;
  if (cs != cudaStreamCaptureStatusActive || !g) return cudaErrorStreamCaptureInvalidated;
  cudaGraphConditionalHandle cond = 0;
  e = cudaGraphConditionalHandleCreate(&cond, g, 0u, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) return e;
  launch_plain(k_retry_arm, 1u, 32, 0, true, st, m, max_iter, cond, 1);
  const cudaGraphNode_t *deps = nullptr;
  const cudaGraphEdgeData *edges = nullptr;
  size_t ndeps = 0;
  e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, &edges, &ndeps);
  if (e != cudaSuccess) return e;
  cudaGraphNodeParams p = {};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = cond;
  p.conditional.type = cudaGraphCondTypeIf;
  p.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  e = cudaGraphAddNode(&node, g, deps, edges, ndeps, &p);
  if (e != cudaSuccess) return e;
  cudaGraph_t body = p.conditional.phGraph_out[0];
  e = cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
  if (e != cudaSuccess) return e;
  e = cudaStreamBeginCaptureToGraph(if_st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  const cudaError_t eb = launch_retry_body<NB>(m, r, x, max_iter, tol, if_st, body_st, pdl);
  const cudaError_t el = cudaPeekAtLastError();
  cudaGraph_t out = nullptr;
  e = cudaStreamEndCapture(if_st, &out);
  return eb != cudaSuccess ? eb : el != cudaSuccess ? el : e;
}

}  // namespace

// Columns of the coupling vectors (nr rounded up to the register chunk).
static int coupling_ldc(int nr) { return (nr + cx::RC - 1) / cx::RC * cx::RC; }

// cmode: 0 = the FP32-based root (no coupling buffers), 1 = automatic,
// 2 = always refine the coupling columns. ff: float-float residual buffers.
size_t mixed_bytes(int S, int N, int nb, int nr, int cmode, int ff) {
  const size_t SN = (size_t)S * N, b2 = (size_t)nb * nb, n = SN * nb + nr;
  size_t t = 0;
  t += align_up(SN * b2 * sizeof(float), 256) * 5;          // Ld Ll Lr Dt W
  t += align_up(SN * nb * sizeof(float), 256) * 3;          // invd y zt
  t += align_up((size_t)S * nr * nb * sizeof(double), 256); // F
  t += align_up((size_t)S * nr * nr * sizeof(double), 256); // U
  t += align_up((size_t)nr * nr * sizeof(double), 256) * 2; // LR Rt
  t += align_up((size_t)nr * sizeof(double) * (cmode && S < 152 * 8 ? 152 * 8 : S), 256);  // tb (grid parts <= max(1216, nr <= 64))
  t += align_up((size_t)nr * sizeof(double), 256);          // d0
  t += align_up(n * sizeof(double), 256);                   // rho
  t += align_up(sizeof(IRCtl), 256);
  if (cmode) {
    const int ldc = coupling_ldc(nr);
    const size_t xb = align_up(SN * nb * ldc * sizeof(float), 256);
    t += xb;                          // Xa
    if (ldc > nb) t += 2 * xb;        // Yb, Zr (else they reuse W and Dt)
  }
  if (ff) {
    t += align_up(SN * b2 * sizeof(float), 256) * 2;                        // Kdh Kdl
    t += align_up((size_t)S * (N > 1 ? N - 1 : 0) * b2 * sizeof(float), 256) * 2;  // Keh Kel
    t += align_up(SN * nb * sizeof(float), 256) * 2;                        // xh xl
  }
  return t;
}

size_t mixed_bytes(int S, int N, int nb, int nr) { return mixed_bytes(S, N, nb, nr, 0, 0); }

// Whether a handle with tolerance tol computes float-float residuals.
bool mixed_ff_residual(double tol, unsigned flags) {
  return !(flags & BM_FLAG_RESIDUAL_FP64) && tol >= mx::kFFMinTol;
}

bool mixed_ffres(const MixedState *m) { return m->ffres != 0; }


cudaError_t mixed_prepare(int nb, int nr) {
  (void)nr;
  if (!tail_nb_supported(nb)) return cudaErrorInvalidValue;
  static std::mutex mu;
  static bool done[64] = {false};
  std::lock_guard<std::mutex> lock(mu);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return cudaErrorUnknown;
  if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
  cudaError_t e = tail_factor_prepare();
  if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
  return e;
}

MixedState *mixed_create(int S, int N, int nb, int nr, int cmode, int ff, void *base, size_t bytes,
                         Status *status, unsigned *tickets, cudaStream_t init_stream, bool sync_init) {
  if (bytes < mixed_bytes(S, N, nb, nr, cmode, ff)) return nullptr;
  MixedState *m = new (std::nothrow) MixedState();
  if (!m) return nullptr;
  m->S = S; m->N = N; m->nb = nb; m->nr = nr; m->Lc = chain_levels(N);
  char *p = (char *)base;
  auto take = [&](size_t b) {
    void *q = p;
    p += align_up(b, 256);
    return q;
  };
  const size_t SN = (size_t)S * N, b2 = (size_t)nb * nb, n = SN * nb + nr;
  m->Ld = (float *)take(SN * b2 * 4); m->Ll = (float *)take(SN * b2 * 4); m->Lr = (float *)take(SN * b2 * 4);
  m->Dt = (float *)take(SN * b2 * 4); m->W = (float *)take(SN * b2 * 4);
  m->invd = (float *)take(SN * nb * 4); m->y = (float *)take(SN * nb * 4); m->zt = (float *)take(SN * nb * 4);
  m->F = (double *)take((size_t)S * nr * nb * 8); m->U = (double *)take((size_t)S * nr * nr * 8);
  m->LR = (double *)take((size_t)nr * nr * 8); m->Rt = (double *)take((size_t)nr * nr * 8);
  m->tb = (double *)take((size_t)nr * 8 * (cmode && S < 152 * 8 ? 152 * 8 : S)); m->d0 = (double *)take((size_t)nr * 8);
  m->rho = (double *)take(n * 8);
  m->ctl = (IRCtl *)take(sizeof(IRCtl));
  m->cmode = cmode;
  m->cxon = &status->coupled;
  if (cmode) {
    m->ldc = coupling_ldc(nr);
    const size_t xb = SN * nb * m->ldc * 4;
    m->Xa = (float *)take(xb);
    m->Xc = m->Xa;
    if (m->ldc > nb) {
      m->Yb = (float *)take(xb);
      m->Zr = (float *)take(xb);
    } else {
      m->Yb = m->W;
      m->Zr = m->Dt;
    }
  }
  if (ff) {
    const size_t ne = (size_t)S * (N > 1 ? N - 1 : 0) * b2;
    m->ffres = 1;
    m->Kdh = (float *)take(SN * b2 * 4); m->Kdl = (float *)take(SN * b2 * 4);
    m->Keh = (float *)take(ne * 4); m->Kel = (float *)take(ne * 4);
    m->xh = (float *)take(SN * nb * 4); m->xl = (float *)take(SN * nb * 4);
  }
  m->status = status;
  m->tickets = tickets;
  if ((sync_init ? cudaMemset(m->ctl, 0, sizeof(IRCtl)) : cudaMemsetAsync(m->ctl, 0, sizeof(IRCtl), init_stream)) !=
      cudaSuccess) {
    delete m;
    return nullptr;
  }
  return m;
}

void mixed_destroy(MixedState *m) { delete m; }

// Root step of the factor, shared with the FP64 path (bm_fp64.cu).
void f64_launch_factor_root_raw(int S, int nr, const double *U, const double *R, double *Rt, double *LR,
                                unsigned *tickets, Status *status, int mode, int *on, cudaStream_t st);
void coupling_launch(const cx::CxView &v, int nb, int *mark, cudaStream_t st);

static cx::CxView cx_view(const MixedState &m, int *on) {
  cx::CxView cv;
  cv.S = m.S; cv.N = m.N; cv.nr = m.nr; cv.ldc = m.ldc; cv.Lc = m.Lc;
  cv.Ld = m.Ld; cv.Ll = m.Ll; cv.Lr = m.Lr; cv.invd = m.invd;
  cv.D = m.D; cv.E = m.E; cv.C = m.C;
  cv.Xa = m.Xa; cv.Yb = m.Yb; cv.Zr = m.Zr; cv.U = m.U;
  cv.on = on;
  return cv;
}

static void launch_ff_split(const MixedState &m, cudaStream_t st) {
  const long n = (long)m.S * (2 * m.N - 1) * m.nb * m.nb;
  long blocks = (n + 1023) / 1024;
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks < 1) blocks = 1;
  switch (m.nb) {
#define X(n)                                                            \
  case n:                                                               \
    launch_plain(k_ff_split<n>, (unsigned)blocks, 256, 0, true, st, m); \
    break;
    BM_TAIL_NB_LIST(X)
#undef X
  }
}

void mixed_launch_factor(MixedState *m, const double *D, const double *E, const double *C, const double *R,
                         cudaStream_t st) {
  m->D = D; m->E = E; m->C = C; m->R = R;
  TailView<float> t{};
  t.S = m->S; t.N = m->N; t.nb = m->nb; t.nr = m->nr; t.Lc = m->Lc;
  t.D = D; t.E = E; t.C = C; t.R = R;
  t.Ld = m->Ld; t.Ll = m->Ll; t.Lr = m->Lr; t.Dt = m->Dt; t.W = m->W; t.invd = m->invd;
  t.F = m->F; t.U = m->U; t.status = m->status;
  // hi + lo planes of K for the float-float residual
  if (m->ffres) launch_ff_split(*m, st);
  tail_factor_launch<float>(t, st);
  int *on = &m->status->coupled;
  if (m->cmode == 0) {
    f64_launch_factor_root_raw(m->S, m->nr, m->U, R, m->Rt, m->LR, m->tickets, m->status, 0, nullptr, st);
    return;
  }
  // automatic mode: the FP32-based root decides whether the coupling
  // columns are refined (and is final when they are not)
  if (m->cmode == 1) {
    launch_plain(k_pivot_spread, (unsigned)m->S, 256, 0, true, st, (const float *)m->invd, m->N, m->nb, m->status);
    f64_launch_factor_root_raw(m->S, m->nr, m->U, R, m->Rt, m->LR, m->tickets, m->status, 1, on, st);
  }
  cx::CxView cv = cx_view(*m, m->cmode == 1 ? on : nullptr);
  coupling_launch(cv, m->nb, m->cmode == 2 ? on : nullptr, st);
  f64_launch_factor_root_raw(m->S, m->nr, m->U, R, m->Rt, m->LR, m->tickets, m->status, m->cmode == 1 ? 2 : 0, on,
                             st);
}


namespace {
// The coupling-column refinement of the resumed solve, gated by *on.
void coupling_launch_cx(const MixedState &m, int *on, cudaStream_t st) {
  coupling_launch(cx_view(m, on), m.nb, nullptr, st);
}
// Its root (Alg. 1 steps 4-5 with the refined U_i), gated by ctl->retry.
void retry_root(const MixedState &m, cudaStream_t st) {
  f64_launch_factor_root_raw(m.S, m.nr, m.U, m.R, m.Rt, m.LR, m.tickets, m.status, 2, &m.ctl->retry, st);
}
}  // namespace

cudaError_t mixed_launch_solve(MixedState *m, const double *r, double *x, int max_refine, double tol,
                               cudaStream_t st, cudaStream_t body_st, cudaStream_t if_st, cudaStream_t body2_st,
                               bool body_pdl) {
  // reset the per-solve control words
  cudaError_t e = cudaMemsetAsync(m->ctl, 0, sizeof(IRCtl), st);
  if (e != cudaSuccess) return e;
  if (m->Xc) {
    switch (m->nb) {
#define X(n)                                                                                          \
  case n:                                                                                             \
    launch_plain(k_mixed_xt<n>, (unsigned)xt_blocks(m->S, m->N, n, m->nr), 256, 0, true, st, *m, r);          \
    break;
      BM_TAIL_NB_LIST(X)
#undef X
    }
  }
  // automatic mode: a refinement that fails without refined coupling
  // columns is resumed with them (k_retry_arm)
  const bool retry = m->cmode == 1;
  if (body_st) {
    switch (m->nb) {
#define X(n)                                                                                  \
  case n:                                                                                     \
    e = capture_loop<n>(*m, r, x, max_refine, tol, st, body_st, body_pdl);                    \
    if (e == cudaSuccess && retry) e = capture_retry<n>(*m, r, x, max_refine, tol, st, if_st, body2_st, body_pdl); \
    return e;
      BM_TAIL_NB_LIST(X)
#undef X
    }
    return cudaErrorInvalidValue;
  }
  for (int it = 0; it <= max_refine; ++it) {
    switch (m->nb) {
#define X(n)                                                     \
  case n:                                                        \
    launch_iteration<n>(*m, r, x, it, max_refine, tol, st, 0, true); \
    break;
      BM_TAIL_NB_LIST(X)
#undef X
    }
  }
  if (retry) {
    launch_plain(k_retry_arm, 1u, 32, 0, true, st, *m, max_refine, (cudaGraphConditionalHandle)0, 0);
    switch (m->nb) {
#define X(n)                                                                        \
  case n:                                                                           \
    launch_retry_body<n>(*m, r, x, max_refine, tol, st, nullptr, true);             \
    break;
      BM_TAIL_NB_LIST(X)
#undef X
    }
  }
  return cudaPeekAtLastError();
}


// rho = r - K x for the last factor's K, float-float or FP64 as the
// refinement of this handle computes it.
void mixed_launch_residual(MixedState *m, const double *r, const double *x, double *rho, cudaStream_t st) {
  MixedState c = *m;
  c.rho = rho;
  const long n = (long)m->S * m->N * m->nb;
  if (m->ffres) {
    long blocks = (n + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    k_x_split<<<(unsigned)blocks, 256, 0, st>>>(c, x);
  }
  const int blocks = xt_blocks(m->S, m->N, m->nb, m->nr);
  switch (m->nb) {
#define X(n)                                                        \
  case n:                                                           \
    k_residual_out<n><<<(unsigned)blocks, 256, 0, st>>>(c, r, x); \
    break;
    BM_TAIL_NB_LIST(X)
#undef X
  }
}

void mixed_launch_export(MixedState *m, double *Ld, double *Ll, double *Lr, double *F, double *LR,
                         cudaStream_t st) {
  const size_t n = (size_t)m->S * m->N * m->nb * m->nb;
  if (Ld) k_widen<<<1024, 256, 0, st>>>(m->Ld, Ld, n);
  if (Ll) k_widen<<<1024, 256, 0, st>>>(m->Ll, Ll, n);
  if (Lr) k_widen<<<1024, 256, 0, st>>>(m->Lr, Lr, n);
  if (F) cudaMemcpyAsync(F, m->F, (size_t)m->S * m->nr * m->nb * sizeof(double), cudaMemcpyDeviceToDevice, st);
  if (LR) cudaMemcpyAsync(LR, m->LR, (size_t)m->nr * m->nr * sizeof(double), cudaMemcpyDeviceToDevice, st);
}

}  // namespace bm
