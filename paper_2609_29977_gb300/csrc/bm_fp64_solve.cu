// FP64 triangular solves (Alg. 2) with one thread-block cluster per tail.
//
// The forward substitution of a tail walks the odd-even levels of
// Gamma_{N-1} upwards and its backward substitution walks them downwards
// (Sec. IV-C); all levels of one tail run inside one launch, the CTAs of
// the tail's cluster splitting the positions of each level and meeting at a
// cluster barrier between levels. Each position is handled by a team of TS
// lanes, one lane per block row: the row's gather of the neighbours'
// contributions is one dependent FMA chain, and the triangular solve with
// the diagonal block passes each new component to the other rows with a
// warp shuffle (through shared memory for teams wider than a warp).
// Values written by other CTAs of the cluster are read with L2-only loads
// after the barrier (release/acquire at cluster scope).
//
// Three launches per solve: tail forward (+ x_1 forward and F_{i,1} y_1),
// the root step (bm_fp64.cu), tail backward (root propagation, x_1, levels).
#include "bm_team.cuh"

namespace bm {
namespace {

__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

template <int NB>
struct SolveCfg {
  static constexpr int TS = NB <= 4 ? 4 : NB <= 8 ? 8 : NB <= 16 ? 16 : NB <= 32 ? 32 : 64;
  static constexpr int THREADS = 256;
  static constexpr int TEAMS = THREADS / TS;
  // CTAs per SM that the register-capped instantiation must allow: with
  // one CTA per tail, four per SM keep up to 608 tails in a single wave on
  // 152 SMs (the uncapped one, 80 registers at nb = 24, fits three)
  static constexpr int MINB = NB <= 32 ? 4 : 2;
};

// Whether a launch of S * CS CTAs needs the register-capped kernels: more
// CTAs than three per SM would otherwise run in a second, mostly empty wave.
inline bool solve_capped(int S, int CS) { return (long)S * CS > 3 * 152; }

// Forward levels of one tail, then x_1: y_1 = L_{i,1}^{-1} z_1 and
// t_i = F_{i,1} y_1. Grid: S * CS CTAs, clusters of CS.
template <int NB, int MINB>
__global__ void __launch_bounds__(256, MINB) k_solve_fwd_tail(F64View v, const double *__restrict__ r, int CS) {
  constexpr int TS = SolveCfg<NB>::TS, TEAMS = SolveCfg<NB>::TEAMS, NB2 = NB * NB;
  __shared__ double sY[TEAMS][NB];
  const Team<TS> tm;
  const int crank = (int)cluster_rank();
  const int s = blockIdx.x / CS;
  const int N = v.N, Lc = v.Lc;
  const size_t sb = (size_t)s * N;
  const int i = tm.lane;   // block row handled by this lane (if < NB)
  pdl_wait();
  for (int lvl = 0; lvl <= Lc; ++lvl) {
    const bool last = lvl == Lc;   // x_1
    const int ntask = last ? 1 : (lvl == 0 ? N / 2 : ((N - 1) >> lvl) + 1);
    for (int t = crank * TEAMS + tm.id; t < ntask; t += CS * TEAMS) {
      int q;
      if (last) q = N;
      else if (lvl == 0) q = 2 * t + 1;
      else {
        const int cnt = (N - 1) >> lvl;
        q = t < cnt ? (t + 1) << lvl : N;
      }
      const bool elim = last || (q < N && ctz32(q) == lvl);
      const size_t zoff = (sb + (N - q)) * NB;
      double z = 0.0;
      if (i < NB) {
        z = (lvl <= 1) ? r[zoff + i] : __ldcg(v.zt + zoff + i);
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
            const double *L = v.Lr + (sb + (N - pl)) * NB2 + i * NB;
            const double *y = v.y + (sb + (N - pl)) * NB;
#pragma unroll
            for (int k = 0; k < NB; ++k) z = fma(-L[k], __ldcg(y + k), z);
          }
          if (pr) {
            const double *L = v.Ll + (sb + (N - pr)) * NB2 + i * NB;
            const double *y = v.y + (sb + (N - pr)) * NB;
#pragma unroll
            for (int k = 0; k < NB; ++k) z = fma(-L[k], __ldcg(y + k), z);
          }
        }
      }
      if (!elim) {
        if (i < NB) v.zt[zoff + i] = z;
        continue;
      }
      // y = L_qq^{-1} z as M w = z, y = inv .* w with the unit lower
      // factor M = L_qq diag(L_qq)^-1, whose row i is column i of the
      // stored block's upper triangle (read coalesced across the lanes)
      const double *Mrow = v.Ld + (sb + (N - q)) * NB2 + (i < NB ? i : 0);
      const double inv = i < NB ? v.invd[zoff + i] : 0.0;
      if (TS <= 32) {
        const int base = (threadIdx.x & 31) & ~(TS - 1);
#pragma unroll
        for (int j = 0; j < NB - 1; ++j) {
          const double wj = __shfl_sync(tm.mask, z, base + j);
          if (i > j && i < NB) z = fma(-Mrow[j * NB], wj, z);
        }
        z *= inv;
        if (i < NB) sY[tm.id][i] = z;
        tm.sync();
      } else {
#pragma unroll
        for (int j = 0; j < NB - 1; ++j) {
          if (i == j) sY[tm.id][j] = z;
          tm.sync();
          if (i > j && i < NB) z = fma(-Mrow[j * NB], sY[tm.id][j], z);
        }
        z *= inv;
        tm.sync();
        if (i < NB) sY[tm.id][i] = z;
      }
      if (i < NB) v.y[zoff + i] = z;
      if (last) {
        tm.sync();
        const int nr = v.nr;
        const double *Fs = v.F + (size_t)s * nr * NB;
        for (int c = i; c < nr; c += TS) {
          double acc = 0.0;
#pragma unroll
          for (int k = 0; k < NB; ++k) acc = fma(Fs[c * NB + k], sY[tm.id][k], acc);
          v.tb[(size_t)s * nr + c] = acc;
        }
      }
      tm.sync();
    }
    cluster_sync();
  }
}

// Backward: root propagation y_1 -= F_{i,1}^T x_0, x_1 = L_{i,1}^{-T} y_1,
// then levels Lc-1..0: x_q = L_qq^{-T}(y_q - L_{a,q}^T x_a - L_{b,q}^T x_b),
// written in natural order.
template <int NB, int MINB>
__global__ void __launch_bounds__(256, MINB) k_solve_bwd_tail(F64View v, double *__restrict__ x, int CS) {
  constexpr int TS = SolveCfg<NB>::TS, TEAMS = SolveCfg<NB>::TEAMS, NB2 = NB * NB;
  __shared__ double sX[TEAMS][NB];
  const Team<TS> tm;
  const int crank = (int)cluster_rank();
  const int s = blockIdx.x / CS;
  const int N = v.N, Lc = v.Lc, nr = v.nr;
  const size_t sb = (size_t)s * N;
  const size_t n0 = (size_t)v.S * N * NB;
  const int i = tm.lane;
  pdl_wait();
  for (int lvl = Lc; lvl >= 0; --lvl) {
    const bool first = lvl == Lc;   // x_1
    const int ntask = first ? 1 : (((N - 1) >> lvl) + 1) / 2;
    for (int t = crank * TEAMS + tm.id; t < ntask; t += CS * TEAMS) {
      const int q = first ? N : (2 * t + 1) << lvl;
      const size_t zoff = (sb + (N - q)) * NB;
      double z = 0.0;
      if (i < NB) {
        z = v.y[zoff + i];
        if (first) {
          const double *Fs = v.F + (size_t)s * nr * NB;
          for (int c = 0; c < nr; ++c) z = fma(-Fs[c * NB + i], __ldcg(x + n0 + c), z);
        } else {
          const int h = 1 << lvl;
          const int a = q - h, b = (q + h <= N - 1) ? q + h : N;
          const double *Lb = v.Lr + (sb + (N - q)) * NB2 + i;
          const double *xb = x + (sb + (N - b)) * NB;
#pragma unroll
          for (int k = 0; k < NB; ++k) z = fma(-Lb[k * NB], __ldcg(xb + k), z);
          if (q > h) {
            const double *La = v.Ll + (sb + (N - q)) * NB2 + i;
            const double *xa = x + (sb + (N - a)) * NB;
#pragma unroll
            for (int k = 0; k < NB; ++k) z = fma(-La[k * NB], __ldcg(xa + k), z);
          }
        }
      }
      // x = L_qq^{-T} z as M^T x = inv .* z with the unit lower factor
      // M = L_qq diag(L_qq)^-1, whose column i is row i of the stored
      // block's upper triangle
      double Mcol[NB];
      const double *Ld = v.Ld + (sb + (N - q)) * NB2 + (i < NB ? i : 0) * NB;
#pragma unroll
      for (int k = 0; k < NB; ++k) Mcol[k] = Ld[k];
      const double inv = i < NB ? v.invd[zoff + i] : 0.0;
      z *= inv;
      if (TS <= 32) {
        const int base = (threadIdx.x & 31) & ~(TS - 1);
#pragma unroll
        for (int j = NB - 1; j > 0; --j) {
          const double xj = __shfl_sync(tm.mask, z, base + j);
          if (i < j) z = fma(-Mcol[j], xj, z);
        }
      } else {
#pragma unroll
        for (int j = NB - 1; j > 0; --j) {
          if (i == j) sX[tm.id][j] = z;
          tm.sync();
          if (i < j) z = fma(-Mcol[j], sX[tm.id][j], z);
        }
      }
      if (i < NB) x[zoff + i] = z;
      tm.sync();
    }
    cluster_sync();
  }
}

int pick_cluster(int S) {
  int cs = 1;
  while (cs < 8 && S * cs * 2 <= 152) cs <<= 1;
  return cs;
}

template <int NB>
cudaError_t launch_tail_kernel(void (*kern)(F64View, const double *, int), const F64View &v, const double *r,
                               cudaStream_t st) {
  const int CS = pick_cluster(v.S);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(v.S * CS));
  cfg.blockDim = dim3(SolveCfg<NB>::THREADS);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, kern, v, r, CS);
}

template <int NB>
cudaError_t launch_bwd_kernel(const F64View &v, double *x, cudaStream_t st) {
  const int CS = pick_cluster(v.S);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(v.S * CS));
  cfg.blockDim = dim3(SolveCfg<NB>::THREADS);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  if (solve_capped(v.S, CS)) return cudaLaunchKernelEx(&cfg, k_solve_bwd_tail<NB, SolveCfg<NB>::MINB>, v, x, CS);
  return cudaLaunchKernelEx(&cfg, k_solve_bwd_tail<NB, 1>, v, x, CS);
}

}  // namespace

void f64_launch_solve_root(const F64View &v, const double *r, double *x, double *r0t, cudaStream_t st);

// The cluster solves substitute with the scaled unit factor that the
// compile-time tail factor stores above each diagonal block's diagonal, so
// they cover exactly the tail factor's block sizes.
#define BM_SOLVE_NB_LIST(X) BM_TAIL_NB_LIST(X)

bool f64_cluster_solve_supported(int nb) {
  switch (nb) {
#define X(n) case n:
    BM_SOLVE_NB_LIST(X)
#undef X
    return true;
  }
  return false;
}

void f64_cluster_launch_solve(const F64View &v, const double *r, double *x, double *r0t, cudaStream_t st) {
  switch (v.nb) {
#define X(n)                                                    \
  case n:                                                       \
    launch_tail_kernel<n>(solve_capped(v.S, pick_cluster(v.S)) ? k_solve_fwd_tail<n, SolveCfg<n>::MINB> \
                                                               : k_solve_fwd_tail<n, 1>, v, r, st); \
    f64_launch_solve_root(v, r, x, r0t, st);                    \
    launch_bwd_kernel<n>(v, x, st);                             \
    break;
    BM_SOLVE_NB_LIST(X)
#undef X
  }
}

}  // namespace bm
