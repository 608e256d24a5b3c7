// FP64 kernels of the two-level factorization (Alg. 1) and triangular
// solves (Alg. 2).
//
// Schedule: one launch per odd-even level of Gamma_{N-1} (Sec. II), one CTA
// per (tail, chain position) task of that level, so scenario-level and
// horizon-level parallelism (Sec. IV, SLP and HLP) both map onto the grid.
// Launch l does, for every position q still in the chain:
//   * the Schur update collected from the level l-1 eliminations next to q
//     (D~_q -= L_{q,p} L_{q,p}^T for the eliminated neighbours p), and
//   * if q belongs to level l: L_qq = chol(D~_q), the coupling blocks
//     L_{b,q} = M_{b,q} L_qq^{-T}, L_{a,q} = M_{a,q} L_qq^{-T} to its right
//     and left neighbours b, a, and the fill coupling between them,
//     M_{b,a} = -L_{b,q} L_{a,q}^T, which becomes a's right coupling.
// Positions eliminated by one launch are never neighbours, every remaining
// position gathers its own update, and every fill block has a single writer,
// so no launch has a write race and no atomics are needed. x_1 (kept last by
// Pi_i, Sec. IV-A) is factored by its own launch, which also forms the
// coupling solve F_{i,1} = C_{i,1} L_{i,1}^{-T} (Theorem 1) and
// U_i = F_{i,1} F_{i,1}^T. The root launch sums R - sum_i U_i in a fixed
// order and the last CTA to finish factors it (Alg. 1, steps 4-5).
//
// GB300 notes: the FP64 pipe retires one warp instruction per 64 cycles per
// SM sub-partition whatever the number of active lanes, so every loop below
// hands out whole output elements across all threads of the CTA (each
// thread's dot product is one dependent FMA chain), and the only
// single-lane FP64 work is the pivot reciprocal square root.
#include <math.h>

#include <mutex>

#include "bm_root.cuh"

namespace bm {
namespace {

__device__ __forceinline__ void cta_copy(double *__restrict__ dst, const double *__restrict__ src, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}
// dst (n x n) := src^T
__device__ __forceinline__ void cta_copy_t(double *__restrict__ dst, const double *__restrict__ src, int n) {
  const int n2 = n * n;
  for (int e = threadIdx.x; e < n2; e += blockDim.x) {
    const int i = e / n, j = e - i * n;
    dst[j * n + i] = src[e];
  }
}
__device__ __forceinline__ void cta_zero(double *dst, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = 0.0;
}
// lower(sD) -= X X^T + Y Y^T (n x n blocks, row-major; X or Y may be null).
__device__ void cta_syrk_sub(double *sD, const double *X, const double *Y, int n) {
  const int ne = n * (n + 1) / 2;
  for (int e = threadIdx.x; e < ne; e += blockDim.x) {
    int i, j;
    tri_ij(e, i, j);
    double acc = sD[i * n + j];
    if (X)
      for (int k = 0; k < n; ++k) acc = fma(-X[i * n + k], X[j * n + k], acc);
    if (Y)
      for (int k = 0; k < n; ++k) acc = fma(-Y[i * n + k], Y[j * n + k], acc);
    sD[i * n + j] = acc;
  }
}

// X (m x n, row stride n) := X L^{-T}, L lower n x n with inverse diagonal inv.
__device__ void cta_trsm_lt(double *X, int m, const double *L, const double *inv, int n) {
  for (int j = 0; j < n; ++j) {
    const double r = inv[j];
    for (int row = threadIdx.x; row < m; row += blockDim.x) X[row * n + j] *= r;
    __syncthreads();
    const int cols = n - j - 1, ne = m * cols;
    for (int e = threadIdx.x; e < ne; e += blockDim.x) {
      const int row = e / cols, k = j + 1 + (e - row * cols);
      X[row * n + k] = fma(-X[row * n + j], L[k * n + j], X[row * n + k]);
    }
    __syncthreads();
  }
}

// Fixed-order CTA sum of one value per thread (blockDim.x a power of two).
__device__ double cta_sum(double v, double *red) {
  red[threadIdx.x] = v;
  for (int w = blockDim.x >> 1; w > 0; w >>= 1) {
    __syncthreads();
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
  }
  __syncthreads();
  const double t = red[0];
  __syncthreads();
  return t;
}

// ---------------------------------------------------------------------------
// Factorization
// ---------------------------------------------------------------------------

__global__ void k_factor_level(F64View v, int lvl) {
  extern __shared__ double sm[];
  __shared__ int sflag;
  const int nb = v.nb, nb2 = nb * nb, N = v.N, s = blockIdx.y;
  const int mb = nb > v.nr ? nb : v.nr;
  double *sD = sm;
  double *sB = sD + mb * mb;   // right coupling, then L_{b,q}
  double *sA = sB + nb2;       // left coupling, then L_{a,q} (stacked under sB)
  double *sInv = sB + (2 * nb2 > v.nr * nb ? 2 * nb2 : v.nr * nb);
  const int q = level_task_pos(N, lvl, blockIdx.x);
  const bool elim = (q < N) && (ctz32(q) == lvl);
  const size_t sb = (size_t)s * N;

  cta_copy(sD, (lvl <= 1 ? v.D : v.Dt) + (sb + (N - q)) * nb2, nb2);
  if (lvl >= 1) {
    const int h = 1 << (lvl - 1);
    int pl = 0, pr = 0;
    if (q < N) {
      pl = q - h;
      if (q + h <= N - 1) pr = q + h;
    } else {
      const int m = ((N - 1) >> (lvl - 1)) << (lvl - 1);
      if (ctz32(m) == lvl - 1) pl = m;
    }
    if (pl) cta_copy(sB, v.Lr + (sb + (N - pl)) * nb2, nb2);
    if (pr) cta_copy(sA, v.Ll + (sb + (N - pr)) * nb2, nb2);
    __syncthreads();
    cta_syrk_sub(sD, pl ? sB : nullptr, pr ? sA : nullptr, nb);
  }
  if (!elim) {
    __syncthreads();
    cta_copy(v.Dt + (sb + (N - q)) * nb2, sD, nb2);
    return;
  }
  __syncthreads();
  if (cta_chol(sD, sInv, nb, &sflag) && threadIdx.x == 0) report_not_spd(v.status, s, N + 1 - q);
  cta_store_lower(v.Ld + (sb + (N - q)) * nb2, sD, nb);
  const int h = 1 << lvl;
  const bool hasA = q > h;
  const int a = q - h;
  // M_{b,q}: the original coupling A_{q+1,q} = E^T at level 0 (and for the
  // last chain position, whose right neighbour is always x_1), else the fill
  // block left by the previous level.
  if (lvl == 0 || q == N - 1)
    cta_copy_t(sB, v.E + ((size_t)s * (N - 1) + (N - q - 1)) * nb2, nb);
  else
    cta_copy(sB, v.W + (sb + (N - q)) * nb2, nb2);
  if (hasA) {
    if (lvl == 0)
      cta_copy(sA, v.E + ((size_t)s * (N - 1) + (N - q)) * nb2, nb2);   // A_{q-1,q}
    else
      cta_copy_t(sA, v.W + (sb + (N - a)) * nb2, nb);                  // M_{q,a}^T
  }
  __syncthreads();
  cta_trsm_lt(sB, hasA ? 2 * nb : nb, sD, sInv, nb);
  cta_copy(v.Lr + (sb + (N - q)) * nb2, sB, nb2);
  if (hasA) {
    cta_copy(v.Ll + (sb + (N - q)) * nb2, sA, nb2);
    double *Wa = v.W + (sb + (N - a)) * nb2;   // becomes M_{b,a}
    for (int e = threadIdx.x; e < nb2; e += blockDim.x) {
      const int i = e / nb, j = e - i * nb;
      double acc = 0.0;
      for (int k = 0; k < nb; ++k) acc = fma(-sB[i * nb + k], sA[j * nb + k], acc);
      Wa[e] = acc;
    }
  } else {
    cta_zero(v.Ll + (sb + (N - q)) * nb2, nb2);
  }
  for (int i = threadIdx.x; i < nb; i += blockDim.x) v.invd[(sb + (N - q)) * nb + i] = sInv[i];
}

// x_1: last Schur update, L_{i,1}, F_{i,1} = C_{i,1} L_{i,1}^{-T}, U_i.
__global__ void k_factor_x1(F64View v) {
  extern __shared__ double sm[];
  __shared__ int sflag;
  const int nb = v.nb, nb2 = nb * nb, N = v.N, nr = v.nr, s = blockIdx.x, Lc = v.Lc;
  const int mb = nb > nr ? nb : nr;
  double *sD = sm, *sB = sD + mb * mb;
  double *sInv = sB + (2 * nb2 > nr * nb ? 2 * nb2 : nr * nb);
  const size_t sb = (size_t)s * N;
  cta_copy(sD, (Lc <= 1 ? v.D : v.Dt) + sb * nb2, nb2);
  if (Lc >= 1) {
    const int m = 1 << (Lc - 1);
    cta_copy(sB, v.Lr + (sb + (N - m)) * nb2, nb2);
    __syncthreads();
    cta_syrk_sub(sD, sB, nullptr, nb);
  }
  __syncthreads();
  if (cta_chol(sD, sInv, nb, &sflag) && threadIdx.x == 0) report_not_spd(v.status, s, 1);
  cta_store_lower(v.Ld + sb * nb2, sD, nb);
  cta_zero(v.Ll + sb * nb2, nb2);
  cta_zero(v.Lr + sb * nb2, nb2);
  for (int i = threadIdx.x; i < nb; i += blockDim.x) v.invd[sb * nb + i] = sInv[i];
  cta_copy(sB, v.C + (size_t)s * nr * nb, nr * nb);
  __syncthreads();
  cta_trsm_lt(sB, nr, sD, sInv, nb);
  cta_copy(v.F + (size_t)s * nr * nb, sB, nr * nb);
  double *Us = v.U + (size_t)s * nr * nr;
  for (int e = threadIdx.x; e < nr * nr; e += blockDim.x) {
    const int i = e / nr, j = e - i * nr;
    double acc = 0.0;
    for (int k = 0; k < nb; ++k) acc = fma(sB[i * nb + k], sB[j * nb + k], acc);
    Us[e] = acc;
  }
}

// Automatic mode of the mixed path: the coupling columns are refined when
// the FP32-based root cannot be trusted. R~ = R - sum_i U_i loses the
// digits of its cancellation gamma = max_j R_jj / R~_jj, and FP32 tails
// give each U_i to about 2^-24 times their conditioning, which the FP32
// factor's pivot spread rho = (max_j L_jj / min_j L_jj)^2 (per tail, max
// over tails) bounds from below. Measured on the workloads (GB300 and the
// oracle's factors): gamma * rho * 2^-24 is about 0.3-0.5 on the medium
// workload and 4-9 on the large serving request, whose FP32-based roots
// converge in 2-3 corrections, and 30-65 on the 10^+-6 mixed workload,
// whose FP32-based root is indefinite or makes refinement diverge.
constexpr double kRootEngage = 16.0;

// Root: R~ = R - sum_i U_i (one warp per lower-triangle entry, fixed
// summation order root_sum_warp), then L_R = chol(R~) by the last CTA to
// finish (Alg. 1, steps 4-5).
//  mode 0: plain.
//  mode 1: probe of the mixed path's automatic mode, with FP32-based U_i:
//          when the Cholesky fails or gamma * rho * 2^-24 > kRootEngage
//          (rho from the status word, left by k_pivot_spread), *on = 1 (the
//          refinement of the coupling columns then runs and a mode-2
//          launch redoes the root) and no failure is reported; else
//          *on = 0 and this is the final root.
//  mode 2: the root after that refinement; returns at once unless *on.
__global__ void __launch_bounds__(256) k_factor_root(F64View v, int mode, int *on) {
  extern __shared__ double sm[];
  __shared__ int last;
  if (mode == 2 && *((volatile const int *)on) == 0) return;
  const int nr = v.nr, ne = nr * (nr + 1) / 2;
  const int e = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (e < ne) root_entry(v.U, v.R, v.S, nr, e, v.Rt);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(&v.tickets[0], 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  double *sR = sm;
  for (int k = threadIdx.x; k < nr * nr; k += blockDim.x) sR[k] = __ldcg(v.Rt + k);
  __syncthreads();
  bool engage = false;
  if (mode == 1) {
    const double rho = (double)__uint_as_float(*((volatile const unsigned *)&v.status->spread));
    const double lim = kRootEngage / (rho * 0x1.0p-24);
    for (int j = 0; j < nr; ++j) {
      const double rt = sR[j * nr + j];
      if (!(rt > 0.0) || v.R[j * nr + j] > lim * rt) engage = true;
    }
  }
  __syncthreads();
  root_chol_store(sR, nr, v.LR, v.status, mode == 1 ? &engage : nullptr, on);
  if (threadIdx.x == 0) v.tickets[0] = 0u;
}

// ---------------------------------------------------------------------------
// Solve (uses the inverse diagonals the factor kept in invd[S][N][nb])
// ---------------------------------------------------------------------------

// y := L^{-1} z in place (L lower n x n in shared memory, inverse diagonal inv).
__device__ void cta_trsv_l(double *z, const double *L, const double *inv, int n) {
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) z[j] *= inv[j];
    __syncthreads();
    for (int k = j + 1 + threadIdx.x; k < n; k += blockDim.x) z[k] = fma(-L[k * n + j], z[j], z[k]);
    __syncthreads();
  }
}
// x := L^{-T} z in place.
__device__ void cta_trsv_lt(double *z, const double *L, const double *inv, int n) {
  for (int j = n - 1; j >= 0; --j) {
    if (threadIdx.x == 0) z[j] *= inv[j];
    __syncthreads();
    for (int k = threadIdx.x; k < j; k += blockDim.x) z[k] = fma(-L[j * n + k], z[j], z[k]);
    __syncthreads();
  }
}

__global__ void k_solve_fwd_level(F64View v, const double *__restrict__ r, int lvl) {
  const double *invd = v.invd;
  extern __shared__ double sm[];
  const int nb = v.nb, nb2 = nb * nb, N = v.N, s = blockIdx.y;
  double *sz = sm, *sL = sm + nb;
  const int q = level_task_pos(N, lvl, blockIdx.x);
  const bool elim = (q < N) && (ctz32(q) == lvl);
  const size_t sb = (size_t)s * N;
  const size_t zoff = (sb + (N - q)) * nb;   // natural stage N+1-q of tail s
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    double z = (lvl <= 1) ? r[zoff + i] : v.zt[zoff + i];
    if (lvl >= 1) {
      const int h = 1 << (lvl - 1);
      int pl = 0, pr = 0;
      if (q < N) {
        pl = q - h;
        if (q + h <= N - 1) pr = q + h;
      } else {
        const int m = ((N - 1) >> (lvl - 1)) << (lvl - 1);
        if (ctz32(m) == lvl - 1) pl = m;
      }
      if (pl) {
        const double *Lb = v.Lr + (sb + (N - pl)) * nb2 + i * nb;
        const double *yp = v.y + (sb + (N - pl)) * nb;
        for (int k = 0; k < nb; ++k) z = fma(-Lb[k], yp[k], z);
      }
      if (pr) {
        const double *Lb = v.Ll + (sb + (N - pr)) * nb2 + i * nb;
        const double *yp = v.y + (sb + (N - pr)) * nb;
        for (int k = 0; k < nb; ++k) z = fma(-Lb[k], yp[k], z);
      }
    }
    sz[i] = z;
  }
  if (!elim) {
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += blockDim.x) v.zt[zoff + i] = sz[i];
    return;
  }
  cta_copy(sL, v.Ld + (sb + (N - q)) * nb2, nb2);
  __syncthreads();
  cta_trsv_l(sz, sL, invd + zoff, nb);
  for (int i = threadIdx.x; i < nb; i += blockDim.x) v.y[zoff + i] = sz[i];
}

// x_1 forward: last update, y_1 = L_{i,1}^{-1} z, t_i = F_{i,1} y_1.
__global__ void k_solve_x1_fwd(F64View v, const double *__restrict__ r) {
  const double *invd = v.invd;
  extern __shared__ double sm[];
  const int nb = v.nb, nb2 = nb * nb, N = v.N, nr = v.nr, s = blockIdx.x, Lc = v.Lc;
  double *sz = sm, *sL = sm + nb;
  const size_t sb = (size_t)s * N;
  const size_t zoff = sb * nb;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    double z = (Lc <= 1) ? r[zoff + i] : v.zt[zoff + i];
    if (Lc >= 1) {
      const int m = 1 << (Lc - 1);
      const double *Lb = v.Lr + (sb + (N - m)) * nb2 + i * nb;
      const double *yp = v.y + (sb + (N - m)) * nb;
      for (int k = 0; k < nb; ++k) z = fma(-Lb[k], yp[k], z);
    }
    sz[i] = z;
  }
  cta_copy(sL, v.Ld + sb * nb2, nb2);
  __syncthreads();
  cta_trsv_l(sz, sL, invd + zoff, nb);
  for (int i = threadIdx.x; i < nb; i += blockDim.x) v.y[zoff + i] = sz[i];
  const double *Fs = v.F + (size_t)s * nr * nb;
  for (int i = threadIdx.x; i < nr; i += blockDim.x) {
    double acc = 0.0;
    for (int k = 0; k < nb; ++k) acc = fma(Fs[i * nb + k], sz[k], acc);
    v.tb[(size_t)s * nr + i] = acc;
  }
}

// Root: r~_0 = r_0 - sum_i t_i (one CTA per component, fixed order); the
// last CTA solves L_R L_R^T x_0 = r~_0 and writes x_0.
__global__ void k_solve_root(F64View v, const double *__restrict__ r, double *__restrict__ x,
                             double *__restrict__ r0t) {
  __shared__ double red[256];
  __shared__ double sR[64 * 64 + 64 + 64];
  __shared__ int last;
  const int nr = v.nr, S = v.S, i = blockIdx.x;
  const size_t n0 = (size_t)S * v.N * v.nb;
  double acc = 0.0;
  for (int s = threadIdx.x; s < S; s += blockDim.x) acc += v.tb[(size_t)s * nr + i];
  const double tot = cta_sum(acc, red);
  if (threadIdx.x == 0) {
    r0t[i] = r[n0 + i] - tot;
    __threadfence();
    last = (atomicAdd(&v.tickets[1], 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double *sL = sR, *sz = sR + nr * nr, *sInv = sz + nr;
  for (int e = threadIdx.x; e < nr * nr; e += blockDim.x) sL[e] = __ldcg(v.LR + e);
  for (int e = threadIdx.x; e < nr; e += blockDim.x) sz[e] = __ldcg(r0t + e);
  __syncthreads();
  for (int e = threadIdx.x; e < nr; e += blockDim.x) sInv[e] = 1.0 / sL[e * nr + e];
  __syncthreads();
  cta_trsv_l(sz, sL, sInv, nr);
  cta_trsv_lt(sz, sL, sInv, nr);
  for (int e = threadIdx.x; e < nr; e += blockDim.x) x[n0 + e] = sz[e];
  if (threadIdx.x == 0) v.tickets[1] = 0u;
}

// Root propagation y_1 -= F_{i,1}^T x_0 and x_1 = L_{i,1}^{-T} y_1.
__global__ void k_solve_x1_bwd(F64View v, double *__restrict__ x) {
  const double *invd = v.invd;
  extern __shared__ double sm[];
  const int nb = v.nb, nb2 = nb * nb, N = v.N, nr = v.nr, s = blockIdx.x;
  double *sz = sm, *sL = sm + nb;
  const size_t sb = (size_t)s * N;
  const size_t n0 = (size_t)v.S * N * nb;
  const double *Fs = v.F + (size_t)s * nr * nb;
  for (int k = threadIdx.x; k < nb; k += blockDim.x) {
    double z = v.y[sb * nb + k];
    for (int i = 0; i < nr; ++i) z = fma(-Fs[i * nb + k], x[n0 + i], z);
    sz[k] = z;
  }
  cta_copy(sL, v.Ld + sb * nb2, nb2);
  __syncthreads();
  cta_trsv_lt(sz, sL, invd + sb * nb, nb);
  for (int i = threadIdx.x; i < nb; i += blockDim.x) x[sb * nb + i] = sz[i];
}

// Backward substitution of level l: x_q = L_qq^{-T} (y_q - L_{a,q}^T x_a - L_{b,q}^T x_b).
__global__ void k_solve_bwd_level(F64View v, double *__restrict__ x, int lvl) {
  const double *invd = v.invd;
  extern __shared__ double sm[];
  const int nb = v.nb, nb2 = nb * nb, N = v.N, s = blockIdx.y;
  double *sz = sm, *sL = sm + nb;
  const int h = 1 << lvl;
  const int q = (2 * blockIdx.x + 1) << lvl;
  const int a = q - h, b = (q + h <= N - 1) ? q + h : N;
  const size_t sb = (size_t)s * N;
  const double *La = v.Ll + (sb + (N - q)) * nb2, *Lb = v.Lr + (sb + (N - q)) * nb2;
  const double *xa = x + (sb + (N - a)) * nb, *xb = x + (sb + (N - b)) * nb;
  for (int k = threadIdx.x; k < nb; k += blockDim.x) {
    double z = v.y[(sb + (N - q)) * nb + k];
    for (int i = 0; i < nb; ++i) z = fma(-Lb[i * nb + k], xb[i], z);
    if (q > h)
      for (int i = 0; i < nb; ++i) z = fma(-La[i * nb + k], xa[i], z);
    sz[k] = z;
  }
  cta_copy(sL, v.Ld + (sb + (N - q)) * nb2, nb2);
  __syncthreads();
  cta_trsv_lt(sz, sL, invd + (sb + (N - q)) * nb, nb);
  for (int i = threadIdx.x; i < nb; i += blockDim.x) x[(sb + (N - q)) * nb + i] = sz[i];
}

}  // namespace

// ---------------------------------------------------------------------------
// Host-side launchers (stream-ordered; called directly or under capture)
// ---------------------------------------------------------------------------

static int factor_threads(int nb) { return nb <= 8 ? 32 : nb <= 16 ? 64 : nb <= 32 ? 128 : 256; }
static int solve_threads(int nb) { return nb <= 32 ? 32 : 64; }

size_t f64_factor_smem(int nb, int nr) {
  const int mb = nb > nr ? nb : nr;
  const size_t b2 = 2 * (size_t)nb * nb > (size_t)nr * nb ? 2 * (size_t)nb * nb : (size_t)nr * nb;
  return ((size_t)mb * mb + b2 + mb) * sizeof(double);
}

bool f64_cluster_solve_supported(int nb);
void f64_cluster_launch_solve(const F64View &v, const double *r, double *x, double *r0t, cudaStream_t st);

// The dynamic shared-memory limit is a per-kernel attribute shared by every
// handle in the process, so it is always raised to what the largest
// supported blocks (nb = nr = 64) need; a handle with small blocks must not
// lower it under another handle's feet.
cudaError_t f64_prepare(int nb, int nr) {
  (void)nb;
  (void)nr;
  static std::mutex mu;
  static bool done[64] = {false};
  std::lock_guard<std::mutex> lock(mu);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return cudaErrorUnknown;
  if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
  nb = nr = 64;
  const int smem = (int)f64_factor_smem(nb, nr);
  cudaError_t e = cudaFuncSetAttribute(k_factor_level, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_factor_x1, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int ssm = (int)(((size_t)nb * nb + nb) * sizeof(double));
  for (const void *f : {(const void *)k_solve_fwd_level, (const void *)k_solve_x1_fwd,
                        (const void *)k_solve_x1_bwd, (const void *)k_solve_bwd_level}) {
    e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, ssm);
    if (e != cudaSuccess) return e;
  }
  e = cudaFuncSetAttribute(k_factor_root, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(((size_t)nr * nr + nr) * sizeof(double)));
  if (e != cudaSuccess) return e;
  e = tail_factor_prepare();
  if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;   // only once everything was set
  return e;
}

// Block sizes with compile-time kernels (bm_tail_factor.cuh) use those; any
// other nb runs the runtime-size kernels above.
static TailView<double> tail_view_of(const F64View &v) {
  TailView<double> t{};
  t.S = v.S; t.N = v.N; t.nb = v.nb; t.nr = v.nr; t.Lc = v.Lc;
  t.D = v.D; t.E = v.E; t.C = v.C; t.R = v.R;
  t.Ld = v.Ld; t.Ll = v.Ll; t.Lr = v.Lr; t.Dt = v.Dt; t.W = v.W; t.invd = v.invd;
  t.F = v.F; t.U = v.U; t.status = v.status;
  t.Rt = v.Rt; t.LR = v.LR; t.tickets = v.tickets;
  return t;
}

// Tunes the tail factor's launch schedule on v's inputs (synchronizes st).
bool f64_tune(const F64View &v, cudaStream_t st, TailSched *out) {
  return tail_factor_tune(tail_view_of(v), st, out);
}

// Part of the FP64 factor for pipelined callers (block sizes with
// compile-time kernels): the grid-wide levels [lo, hi) of tails [s0, s1)
// and, if top, the top kernel over those tails; its last CTA does the root
// step only when the range holds every tail.
void f64_launch_factor_part(const F64View &v, int s0, int s1, int lo, int hi, bool top, cudaStream_t st,
                            const TailSched *sc) {
  TailView<double> t = tail_view_of(v);
  const size_t o = (size_t)s0 * v.N, b2 = (size_t)v.nb * v.nb;
  t.S = s1 - s0;
  t.s0 = s0;
  t.D = v.D + o * b2;
  t.E = v.E ? v.E + (size_t)s0 * (v.N - 1) * b2 : nullptr;
  t.C = v.C + (size_t)s0 * v.nr * v.nb;
  t.Ld = v.Ld + o * b2; t.Ll = v.Ll + o * b2; t.Lr = v.Lr + o * b2;
  t.Dt = v.Dt + o * b2; t.W = v.W + o * b2;
  t.invd = v.invd + o * v.nb;
  t.F = v.F + (size_t)s0 * v.nr * v.nb;
  t.U = v.U + (size_t)s0 * v.nr * v.nr;
  if (s0 != 0 || s1 != v.S) t.LR = nullptr;
  tail_factor_launch_range(t, st, sc, lo, hi, top);
}

void f64_launch_factor(const F64View &v, cudaStream_t st, const TailSched *sc) {
  if (tail_nb_supported(v.nb)) {
    // the top kernel's last CTA finishes with the root step
    tail_factor_launch<double>(tail_view_of(v), st, sc);
    return;
  } else {
    const int T = factor_threads(v.nb);
    const size_t smem = f64_factor_smem(v.nb, v.nr);
    for (int l = 0; l < v.Lc; ++l) {
      dim3 grid(level_tasks(v.N, l), v.S);
      k_factor_level<<<grid, T, smem, st>>>(v, l);
    }
    k_factor_x1<<<v.S, T, smem, st>>>(v);
  }
  const int ne = v.nr * (v.nr + 1) / 2;
  k_factor_root<<<(ne + 7) / 8, 256, ((size_t)v.nr * v.nr + v.nr) * sizeof(double), st>>>(v, 0, nullptr);
}

// Root step of the factor for callers that hold raw buffers (mixed path);
// mode and on as for k_factor_root.
void f64_launch_factor_root_raw(int S, int nr, const double *U, const double *R, double *Rt, double *LR,
                                unsigned *tickets, Status *status, int mode, int *on, cudaStream_t st) {
  F64View v{};
  v.S = S;
  v.nr = nr;
  v.U = const_cast<double *>(U);
  v.R = R;
  v.Rt = Rt;
  v.LR = LR;
  v.tickets = tickets;
  v.status = status;
  const int ne = nr * (nr + 1) / 2;
  k_factor_root<<<(ne + 7) / 8, 256, ((size_t)nr * nr + nr) * sizeof(double), st>>>(v, mode, on);
}

// Lower triangles of nblk nb x nb blocks, upper triangles zero (the tail
// factor keeps the scaled unit factor's transpose above the diagonal).
__global__ void k_copy_lower(const double *__restrict__ src, double *__restrict__ dst, long n, int nb) {
  const int nb2 = nb * nb;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    const int w = (int)(e % nb2), i = w / nb, j = w - i * nb;
    dst[e] = j <= i ? src[e] : 0.0;
  }
}

void f64_launch_export_ld(const F64View &v, double *Ld, cudaStream_t st) {
  const long n = (long)v.S * v.N * v.nb * v.nb;
  long blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_copy_lower<<<(unsigned)blocks, 256, 0, st>>>(v.Ld, Ld, n, v.nb);
}

void f64_launch_solve_root(const F64View &v, const double *r, double *x, double *r0t, cudaStream_t st) {
  k_solve_root<<<v.nr, 256, 0, st>>>(v, r, x, r0t);
}

void f64_launch_solve(const F64View &v, const double *r, double *x, double *r0t, cudaStream_t st) {
  if (f64_cluster_solve_supported(v.nb)) {
    f64_cluster_launch_solve(v, r, x, r0t, st);
    return;
  }
  const int T = solve_threads(v.nb);
  const size_t smem = ((size_t)v.nb * v.nb + v.nb) * sizeof(double);
  for (int l = 0; l < v.Lc; ++l) {
    dim3 grid(level_tasks(v.N, l), v.S);
    k_solve_fwd_level<<<grid, T, smem, st>>>(v, r, l);
  }
  k_solve_x1_fwd<<<v.S, T, smem, st>>>(v, r);
  k_solve_root<<<v.nr, 256, 0, st>>>(v, r, x, r0t);
  k_solve_x1_bwd<<<v.S, T, smem, st>>>(v, x);
  for (int l = v.Lc - 1; l >= 0; --l) {
    dim3 grid(level_elims(v.N, l), v.S);
    k_solve_bwd_level<<<grid, T, smem, st>>>(v, x, l);
  }
}

}  // namespace bm
