// Register-resident variant of the tail tasks (Alg. 1, steps 1-3) for block
// sizes up to 32: a team of TS = next power of two >= NB lanes (at most one
// warp) handles one chain position, lane i holding row i of every block it
// works on in registers:
//   * the gathered Schur update D~_q -= X X^T streams the other rows of X
//     from shared memory (broadcast reads),
//   * the Cholesky of D~_q is right-looking with each column's entries
//     exchanged by warp shuffles (no shared memory, no barrier),
//   * the two coupling solves M L^{-T} reuse the shuffled columns of L,
//   * the fill -L_{b,q} L_{a,q}^T streams L_{a,q} from shared memory.
// D~ is kept with both triangles (each lane owns a full row), so the level
// workspace is read back row by row. Used for the FP32 tails of the mixed
// path, where the shared-memory variant is latency-bound.
#pragma once

#include "bm_team.cuh"

namespace bm {
namespace rows {

template <int NB>
struct Cfg {
  static constexpr int TS = NB <= 4 ? 4 : NB <= 8 ? 8 : NB <= 16 ? 16 : 32;
  static constexpr int LD = NB + 1;   // padded row stride of staged blocks (no bank conflicts)
  static constexpr int SM = NB * LD;  // staged block size in elements
};

template <typename T>
__device__ __forceinline__ T shfl(unsigned mask, T v, int src, int width) {
  return __shfl_sync(mask, v, src, width);
}

// NB FP64 values addr(0), ..., addr(NB-1) rounded to FP32, every load of a
// chunk issued before its first conversion. The conversion is the hardware
// round-to-nearest (on this GPU's FP64 pipe, idle in these FP32 tasks; the
// same bits as the integer rounding d2f_rn, which a GPU test checks), so
// that no branch orders the loads: with the integer rounding's
// out-of-range branch after each value, each load waited for the data of
// the one before.
template <typename T, int NB, typename Addr>
__device__ __forceinline__ void load_to_t(T (&dst)[NB], Addr addr) {
  static_assert(sizeof(T) == sizeof(float), "FP32 tasks");
  constexpr int CH = NB <= 32 ? NB : 16;
#pragma unroll
  for (int j0 = 0; j0 < NB; j0 += CH) {
    double v[CH];
#pragma unroll
    for (int t = 0; t < CH; ++t)
      if (j0 + t < NB) v[t] = addr(j0 + t);
#pragma unroll
    for (int t = 0; t < CH; ++t)
      if (j0 + t < NB) dst[j0 + t] = __double2float_rn(v[t]);
  }
}

// Copy an NB x NB block (global, type T) into shared memory with the team
// (row stride Cfg<NB>::LD).
template <typename T, int NB, int TS>
__device__ __forceinline__ void stage(T *__restrict__ s, const T *__restrict__ g, int lane) {
#pragma unroll
  for (int e = lane; e < NB * NB; e += TS) {
    const int r = e / NB, c = e - r * NB;
    s[r * Cfg<NB>::LD + c] = g[e];
  }
}

// d[j] -= sum_k X[i][k] X[j][k] for all j, X staged in sX, row i = lane.
template <typename T, int NB>
__device__ __forceinline__ void syrk_row(T (&d)[NB], const T *__restrict__ sX, int ir) {
  constexpr int LD = Cfg<NB>::LD;
  T xi[NB];
#pragma unroll
  for (int k = 0; k < NB; ++k) xi[k] = sX[ir * LD + k];
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    T acc = T(0);
#pragma unroll
    for (int k = 0; k < NB; ++k) acc = fma_t<T>(xi[k], sX[j * LD + k], acc);
    d[j] -= acc;
  }
}

// Right-looking Cholesky on rows held by lanes (lane i has row i in d[]).
// On return d[j] (j <= i) is L_ij; rinv is 1/L_ii. Returns 1 + the first
// failing column (uniform over the team), 0 if all pivots are positive.
template <typename T, int NB, int TS>
__device__ __forceinline__ int chol_rows(T (&d)[NB], T &rinv, unsigned mask, int i) {
  int fail = 0;
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    T piv = shfl<T>(mask, d[j], j, TS);
    if (!pivot_ok(piv)) {
      if (!fail) fail = j + 1;
      piv = T(1);
    }
    const T r = rsqrt_t<T>(piv);
    if (i == j) {
      d[j] = piv * r;
      rinv = r;
    } else {
      d[j] *= r;
    }
#pragma unroll
    for (int k = j + 1; k < NB; ++k) {
      const T lkj = shfl<T>(mask, d[j], k, TS);
      d[k] = fma_t<T>(-d[j], lkj, d[k]);
    }
  }
  return fail;
}

// b := b L^{-T}, a := a L^{-T} for the rows held by this lane; L is
// distributed by rows over the team (lane k holds L_k* in lk[]).
template <typename T, int NB, int TS, bool TWO>
__device__ __forceinline__ void trsm_rows(T (&b)[NB], T (&a)[NB], const T (&lk)[NB], T rinv, unsigned mask) {
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    const T rj = shfl<T>(mask, rinv, j, TS);
    b[j] *= rj;
    if (TWO) a[j] *= rj;
#pragma unroll
    for (int k = j + 1; k < NB; ++k) {
      const T lkj = shfl<T>(mask, lk[j], k, TS);
      b[k] = fma_t<T>(-b[j], lkj, b[k]);
      if (TWO) a[k] = fma_t<T>(-a[j], lkj, a[k]);
    }
  }
}

// chol_rows and trsm_rows fused column by column: each entry L_kj that
// the Cholesky broadcasts also updates the coupling rows b (and a), which
// trsm_rows would broadcast a second time, and the inverse pivot 1/L_jj is
// the r every lane has just computed. The values and the order of the
// operations on d, b and a are those of chol_rows followed by trsm_rows.
template <typename T, int NB, int TS, bool TWO>
__device__ __forceinline__ int chol_trsm_rows(T (&d)[NB], T (&b)[NB], T (&a)[NB], T &rinv, unsigned mask, int i) {
  int fail = 0;
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    T piv = shfl<T>(mask, d[j], j, TS);
    if (!pivot_ok(piv)) {
      if (!fail) fail = j + 1;
      piv = T(1);
    }
    const T r = rsqrt_t<T>(piv);
    if (i == j) {
      d[j] = piv * r;
      rinv = r;
    } else {
      d[j] *= r;
    }
    b[j] *= r;
    if (TWO) a[j] *= r;
#pragma unroll
    for (int k = j + 1; k < NB; ++k) {
      const T lkj = shfl<T>(mask, d[j], k, TS);
      d[k] = fma_t<T>(-d[j], lkj, d[k]);
      b[k] = fma_t<T>(-b[j], lkj, b[k]);
      if (TWO) a[k] = fma_t<T>(-a[j], lkj, a[k]);
    }
  }
  return fail;
}

// One task of level lvl with register-resident rows.
// FUSED: the Cholesky and the coupling solves in one column loop
// (chol_trsm_rows; the grid-wide level kernel) or one after the other (the
// per-tail top kernel and the batched form, whose register budget the
// fused loop would exceed). Both give the same bits.
template <typename T, int NB, bool FUSED = false>
__device__ __forceinline__ void factor_task_rows(const TailView<T> &v, T *sX, int lane, unsigned mask, int s, int q,
                                                 int lvl, bool elim) {
  constexpr int TS = Cfg<NB>::TS, NB2 = NB * NB;
  const int N = v.N;
  const size_t sb = (size_t)s * N;
  const int i = lane;
  const bool act = i < NB;
  const int ir = act ? i : 0;
  T d[NB];
  if (lvl <= 1) {
    const double *Dq = v.D + (sb + (N - q)) * NB2;
    load_to_t<T, NB>(d, [&](int j) { return j <= ir ? Dq[ir * NB + j] : Dq[j * NB + ir]; });
  } else {
    const T *Dq = v.Dt + (sb + (N - q)) * NB2 + ir * NB;
#pragma unroll
    for (int j = 0; j < NB; ++j) d[j] = Dq[j];
  }
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
      stage<T, NB, TS>(sX, v.Lr + (sb + (N - pl)) * NB2, lane);
      __syncwarp(mask);
      syrk_row<T, NB>(d, sX, ir);
      __syncwarp(mask);
    }
    if (pr) {
      stage<T, NB, TS>(sX, v.Ll + (sb + (N - pr)) * NB2, lane);
      __syncwarp(mask);
      syrk_row<T, NB>(d, sX, ir);
      __syncwarp(mask);
    }
  }
  if (!elim) {
    if (act) {
      T *o = v.Dt + (sb + (N - q)) * NB2 + i * NB;
#pragma unroll
      for (int j = 0; j < NB; ++j) o[j] = d[j];
    }
    return;
  }
  // couplings: rows i of M_{b,q} and M_{a,q}
  const int hh = 1 << lvl;
  const bool hasA = q > hh;
  const int a = q - hh;
  T b[NB], av[NB];
  if (lvl == 0 || q == N - 1) {
    const double *Eb = v.E + ((size_t)s * (N - 1) + (N - q - 1)) * NB2;   // M_{b,q} = E^T
    load_to_t<T, NB>(b, [&](int k) { return Eb[k * NB + ir]; });
  } else {
    const T *Wb = v.W + (sb + (N - q)) * NB2 + ir * NB;
#pragma unroll
    for (int k = 0; k < NB; ++k) b[k] = Wb[k];
  }
  if (hasA) {
    if (lvl == 0) {
      const double *Ea = v.E + ((size_t)s * (N - 1) + (N - q)) * NB2 + ir * NB;
      load_to_t<T, NB>(av, [&](int k) { return Ea[k]; });
    } else {
      const T *Wa = v.W + (sb + (N - a)) * NB2;   // M_{a,q} = W[a]^T
#pragma unroll
      for (int k = 0; k < NB; ++k) av[k] = Wa[k * NB + ir];
    }
  } else {
#pragma unroll
    for (int k = 0; k < NB; ++k) av[k] = T(0);
  }
  T rinv = T(1);
  int fail;
  if constexpr (FUSED) {
    // one instantiation for both cases: without a left neighbour av is zero
    // and stays +0 through the updates
    fail = chol_trsm_rows<T, NB, TS, true>(d, b, av, rinv, mask, i);
  } else {
    fail = chol_rows<T, NB, TS>(d, rinv, mask, i);
    if (hasA)
      trsm_rows<T, NB, TS, true>(b, av, d, rinv, mask);
    else
      trsm_rows<T, NB, TS, false>(b, av, d, rinv, mask);
  }
  if (i == 0 && fail) report_not_spd(v.status, s, N + 1 - q);
  if (act) {
    T *Ld = v.Ld + (sb + (N - q)) * NB2 + i * NB;
    T *Lb = v.Lr + (sb + (N - q)) * NB2 + i * NB;
    T *La = v.Ll + (sb + (N - q)) * NB2 + i * NB;
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      Ld[j] = j <= i ? d[j] : T(0);
      Lb[j] = b[j];
      La[j] = av[j];
    }
    v.invd[(sb + (N - q)) * NB + i] = rinv;
  }
  if (hasA) {
    // fill M_{b,a} = -L_{b,q} L_{a,q}^T: stage the rows of L_{a,q}
    constexpr int LD = Cfg<NB>::LD;
    if (act) {
#pragma unroll
      for (int k = 0; k < NB; ++k) sX[i * LD + k] = av[k];
    }
    __syncwarp(mask);
    if (act) {
      T *Wo = v.W + (sb + (N - a)) * NB2 + i * NB;
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        T acc = T(0);
#pragma unroll
        for (int k = 0; k < NB; ++k) acc = fma_t<T>(b[k], sX[j * LD + k], acc);
        Wo[j] = -acc;
      }
    }
    __syncwarp(mask);
  }
}

// x_1 of tail s: last update and L_{i,1} with register rows, then F_{i,1} =
// C_{i,1} L_{i,1}^{-T} and U_i = F F^T in FP64. sbuf: nr*NB doubles followed
// by NB*NB + NB values of type T.
template <typename T, int NB>
__device__ __forceinline__ void x1_task_rows(const TailView<T> &v, void *sbuf, int lane, unsigned mask, int s) {
  constexpr int TS = Cfg<NB>::TS, NB2 = NB * NB;
  const int N = v.N, nr = v.nr, Lc = v.Lc;
  const size_t sb = (size_t)s * N;
  constexpr int LD = Cfg<NB>::LD;
  double *sC = (double *)sbuf;
  T *sL = (T *)(sC + nr * NB), *sInv = sL + NB * LD;
  const int i = lane;
  const bool act = i < NB;
  const int ir = act ? i : 0;
  T d[NB];
  if (Lc <= 1) {
    const double *Dq = v.D + sb * NB2;
    load_to_t<T, NB>(d, [&](int j) { return j <= ir ? Dq[ir * NB + j] : Dq[j * NB + ir]; });
  } else {
    const T *Dq = v.Dt + sb * NB2 + ir * NB;
#pragma unroll
    for (int j = 0; j < NB; ++j) d[j] = Dq[j];
  }
  if (Lc >= 1) {
    const int m = 1 << (Lc - 1);
    stage<T, NB, TS>(sL, v.Lr + (sb + (N - m)) * NB2, lane);
    __syncwarp(mask);
    syrk_row<T, NB>(d, sL, ir);
    __syncwarp(mask);
  }
  T rinv = T(1);
  const int fail = chol_rows<T, NB, TS>(d, rinv, mask, i);
  if (i == 0 && fail) report_not_spd(v.status, s, 1);
  if (act) {
    T *Ld = v.Ld + sb * NB2 + i * NB;
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      Ld[j] = j <= i ? d[j] : T(0);
      sL[i * LD + j] = j <= i ? d[j] : T(0);
      v.Lr[sb * NB2 + i * NB + j] = T(0);
      v.Ll[sb * NB2 + i * NB + j] = T(0);
    }
    v.invd[sb * NB + i] = rinv;
    sInv[i] = rinv;
  }
  for (int e = lane; e < nr * NB; e += TS) sC[e] = v.C[(size_t)s * nr * NB + e];
  __syncwarp(mask);
  // F = C L^{-T} in FP64, one row of C per lane (column sweep within the row)
  for (int c = lane; c < nr; c += TS) {
    double f[NB];
#pragma unroll
    for (int k = 0; k < NB; ++k) f[k] = sC[c * NB + k];
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      f[j] *= to_d<T>(sInv[j]);
#pragma unroll
      for (int k = j + 1; k < NB; ++k) f[k] = fma(-f[j], to_d<T>(sL[k * LD + j]), f[k]);
    }
#pragma unroll
    for (int k = 0; k < NB; ++k) {
      sC[c * NB + k] = f[k];
      v.F[(size_t)s * nr * NB + c * NB + k] = f[k];
    }
  }
  __syncwarp(mask);
  double *Us = v.U + (size_t)s * nr * nr;
  for (int e = lane; e < nr * nr; e += TS) {
    const int a = e / nr, b = e - a * nr;
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < NB; ++k) acc = fma(sC[a * NB + k], sC[b * NB + k], acc);
    Us[e] = acc;
  }
}

template <typename T, int NB>
__host__ __device__ constexpr size_t x1_rows_bytes(int nr) {
  return (size_t)nr * NB * sizeof(double) + (NB * (NB + 1) + NB) * sizeof(T);
}

}  // namespace rows
}  // namespace bm

namespace bm {
namespace rows {

// Grid-wide level with register rows: tasks of all tails, eliminated
// positions first; TS lanes per task, 128 threads per CTA.
template <typename T, int NB>
__global__ void __launch_bounds__(128, 4) k_level_rows(TailView<T> v, int lvl) {
  constexpr int TS = Cfg<NB>::TS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int team = threadIdx.x / TS, lane = threadIdx.x % TS;
  const unsigned mask = TS == 32 ? 0xffffffffu : (((1u << TS) - 1u) << ((threadIdx.x & 31) / TS * TS));
  T *sX = (T *)smem_raw + team * Cfg<NB>::SM;
  const int N = v.N, S = v.S;
  const int E = level_elims(N, lvl);
  const int G = lvl == 0 ? 0 : ((N - 1) >> (lvl + 1)) + 1;
  const long g = (long)blockIdx.x * (blockDim.x / TS) + team;
  pdl_wait();
  if (g < (long)S * (E + G)) {
    int s, q;
    bool elim;
    if (g < (long)S * E) {
      s = (int)(g / E);
      q = (2 * (int)(g - (long)s * E) + 1) << lvl;
      elim = true;
    } else {
      const long g2 = g - (long)S * E;
      s = (int)(g2 / G);
      const int j = (int)(g2 - (long)s * G);
      q = j < G - 1 ? (j + 1) << (lvl + 1) : N;
      elim = false;
    }
    factor_task_rows<T, NB, true>(v, sX, lane, mask, s, q, lvl, elim);
  }
  pdl_trigger();
}

// Top levels lvl0..Lc-1 and x_1 of one tail per CTA (four teams).
template <typename T, int NB>
__global__ void __launch_bounds__(128) k_top_rows(TailView<T> v, int lvl0) {
  constexpr int TS = Cfg<NB>::TS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int team = threadIdx.x / TS, lane = threadIdx.x % TS, teams = blockDim.x / TS;
  const unsigned mask = TS == 32 ? 0xffffffffu : (((1u << TS) - 1u) << ((threadIdx.x & 31) / TS * TS));
  T *sX = (T *)smem_raw + team * Cfg<NB>::SM;
  const int N = v.N, s = blockIdx.x;
  pdl_wait();
  for (int lvl = lvl0; lvl < v.Lc; ++lvl) {
    const int E = level_elims(N, lvl);
    const int G = lvl == 0 ? 0 : ((N - 1) >> (lvl + 1)) + 1;
    for (int t = team; t < E + G; t += teams) {
      const bool elim = t < E;
      const int q = elim ? (2 * t + 1) << lvl : (t - E < G - 1 ? (t - E + 1) << (lvl + 1) : N);
      factor_task_rows<T, NB>(v, sX, lane, mask, s, q, lvl, elim);
    }
    __syncthreads();
  }
  if (team == 0) x1_task_rows<T, NB>(v, smem_raw, lane, mask, s);
  pdl_trigger();
}

template <typename T, int NB>
cudaError_t prepare_rows() {
  cudaError_t e = cudaFuncSetAttribute(k_level_rows<T, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_top_rows<T, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
}

template <typename T, int NB>
void launch_tail_rows(const TailView<T> &v, cudaStream_t st) {
  constexpr int TS = Cfg<NB>::TS;
  const int Tl = top_level(v.N);
  const int tpc = 128 / TS;
  for (int l = 0; l < Tl; ++l) {
    const int E = level_elims(v.N, l);
    const int G = l == 0 ? 0 : ((v.N - 1) >> (l + 1)) + 1;
    const long tasks = (long)v.S * (E + G);
    const long blocks = (tasks + tpc - 1) / tpc;
    launch_pdl(k_level_rows<T, NB>, (unsigned)blocks, 128, (size_t)tpc * Cfg<NB>::SM * sizeof(T), st, v, l);
  }
  const int teams = 4;
  size_t smem = (size_t)teams * Cfg<NB>::SM * sizeof(T);
  const size_t x1b = x1_rows_bytes<T, NB>(v.nr);
  if (x1b > smem) smem = x1b;
  launch_pdl(k_top_rows<T, NB>, (unsigned)v.S, teams * TS, smem, st, v, Tl);
}

}  // namespace rows
}  // namespace bm

// ---------------------------------------------------------------------------
// Wide variant for 32 < NB <= 64: a team of 64 lanes (two warps, named
// barrier per team), lane i holding row i. Columns of the Cholesky factor
// are exchanged through shared memory (two barriers per column); the
// triangular solves read the finished factor from shared memory.
// ---------------------------------------------------------------------------
namespace bm {
namespace rows {

template <int NB>
struct WCfg {
  static constexpr int TS = 64;
  // row stride of staged blocks: a multiple of 4 floats, so that rows are
  // read with 16-byte loads, and 52 mod 32 = 20, so that the eight lanes of
  // one 16-byte wavefront hit distinct bank groups when they read their own rows
  static constexpr int LD = (NB + 3) / 4 * 4 + 4;
  static constexpr int SM = NB * LD;
  // per-team shared memory (elements of T): staged block, factor (stored
  // by columns), two column buffers, two pivot slots and padding to 16 bytes
  static constexpr int ELEMS = 2 * SM + 2 * NB + 4;
  static_assert(NB % 4 == 0, "the wide variant reads blocks as groups of four");
};

__device__ __forceinline__ void team_bar(int id) { asm volatile("bar.sync %0, 64;" ::"r"(id) : "memory"); }

// Four consecutive floats of shared memory (16-byte aligned).
__device__ __forceinline__ float4 lds4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ float f4at(const float4 &v, int e) { return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w; }

// Copy an NB x NB float block (global, contiguous) into shared memory with
// row stride LD, four floats per access.
template <typename T, int NB>
__device__ __forceinline__ void stage_w(T *__restrict__ s, const T *__restrict__ g, int lane) {
  static_assert(sizeof(T) == 4, "wide variant is FP32");
  constexpr int LD = WCfg<NB>::LD, Q = NB * NB / 4;
  const float4 *g4 = reinterpret_cast<const float4 *>(g);
#pragma unroll
  for (int e = lane; e < Q; e += 64) {
    const int r = (4 * e) / NB, c = 4 * e - r * NB;
    *reinterpret_cast<float4 *>(s + r * LD + c) = g4[e];
  }
}

// Right-looking Cholesky on lane-owned rows with shared-memory exchange:
// lane j publishes the pivot, every lane scales its entry of column j and
// publishes it, then every lane updates its row from the column (read four
// entries at a time).
template <typename T, int NB>
__device__ __forceinline__ int chol_rows_w(T (&d)[NB], T &rinv, int i, T *sCol, T *sPiv, int bar) {
  int fail = 0;
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    T *col = sCol + (j & 1) * NB;
    if (i == j) sPiv[j & 1] = d[j];
    team_bar(bar);
    T piv = sPiv[j & 1];
    if (!pivot_ok(piv)) {
      if (!fail) fail = j + 1;
      piv = T(1);
    }
    const T r = rsqrt_t<T>(piv);
    if (i == j) {
      d[j] = piv * r;
      rinv = r;
    } else {
      d[j] *= r;
    }
    if (i < NB) col[i] = d[j];
    team_bar(bar);
#pragma unroll
    for (int g = (j + 1) / 4; g < NB / 4; ++g) {
      const float4 v = lds4(col + 4 * g);
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (4 * g + e > j) d[4 * g + e] = fma_t<T>(-d[j], f4at(v, e), d[4 * g + e]);
    }
  }
  return fail;
}

// x := x L^{-T} for a lane-owned row; the factor is staged by columns
// (sLt[j * LD + k] = L_kj), sInv holds 1 / L_jj.
template <typename T, int NB>
__device__ __forceinline__ void trsm_row_w(T (&x)[NB], const T *sLt, const T *sInv) {
  constexpr int LD = WCfg<NB>::LD;
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    x[j] *= sInv[j];
#pragma unroll
    for (int g = (j + 1) / 4; g < NB / 4; ++g) {
      const float4 v = lds4(sLt + j * LD + 4 * g);
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (4 * g + e > j) x[4 * g + e] = fma_t<T>(-x[j], f4at(v, e), x[4 * g + e]);
    }
  }
}

// acc_j = sum_k a[k] X[j][k] for every row j of the staged block, each row
// read four entries at a time; out[j] = sign * acc_j (+ out[j] if ADD).
template <typename T, int NB, bool ADD>
__device__ __forceinline__ void rowdot_w(T (&out)[NB], const T (&a)[NB], const T *__restrict__ sX, T sign) {
  constexpr int LD = WCfg<NB>::LD;
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    T acc = T(0);
#pragma unroll
    for (int g = 0; g < NB / 4; ++g) {
      const float4 v = lds4(sX + j * LD + 4 * g);
      acc = fma_t<T>(a[4 * g + 0], v.x, acc);
      acc = fma_t<T>(a[4 * g + 1], v.y, acc);
      acc = fma_t<T>(a[4 * g + 2], v.z, acc);
      acc = fma_t<T>(a[4 * g + 3], v.w, acc);
    }
    out[j] = ADD ? out[j] + sign * acc : sign * acc;
  }
}

// d[j] -= sum_k X[i][k] X[j][k] for all j, X staged in sX, row i = lane.
template <typename T, int NB>
__device__ __forceinline__ void syrk_row_w(T (&d)[NB], const T *__restrict__ sX, int ir) {
  constexpr int LD = WCfg<NB>::LD;
  T xi[NB];
#pragma unroll
  for (int g = 0; g < NB / 4; ++g) {
    const float4 v = lds4(sX + ir * LD + 4 * g);
    xi[4 * g] = v.x;
    xi[4 * g + 1] = v.y;
    xi[4 * g + 2] = v.z;
    xi[4 * g + 3] = v.w;
  }
  rowdot_w<T, NB, true>(d, xi, sX, T(-1));
}

// Row ir of a float block row (16-byte aligned) into registers.
template <typename T, int NB>
__device__ __forceinline__ void load_row4(T (&d)[NB], const T *__restrict__ row) {
  const float4 *r4 = reinterpret_cast<const float4 *>(row);
#pragma unroll
  for (int g = 0; g < NB / 4; ++g) {
    const float4 v = r4[g];
    d[4 * g] = v.x;
    d[4 * g + 1] = v.y;
    d[4 * g + 2] = v.z;
    d[4 * g + 3] = v.w;
  }
}
template <typename T, int NB>
__device__ __forceinline__ void store_row4(T *__restrict__ row, const T (&d)[NB]) {
  float4 *r4 = reinterpret_cast<float4 *>(row);
#pragma unroll
  for (int g = 0; g < NB / 4; ++g) r4[g] = make_float4(d[4 * g], d[4 * g + 1], d[4 * g + 2], d[4 * g + 3]);
}

// One task of level lvl, wide team (sbuf: WCfg<NB>::ELEMS elements of T).
template <typename T, int NB>
__device__ __forceinline__ void factor_task_rows_w(const TailView<T> &v, T *sbuf, int lane, int bar, int s, int q,
                                                   int lvl, bool elim) {
  constexpr int NB2 = NB * NB, LD = WCfg<NB>::LD, SM = WCfg<NB>::SM;
  T *sX = sbuf, *sL = sbuf + SM, *sCol = sL + SM, *sPiv = sCol + 2 * NB;
  const int N = v.N;
  const size_t sb = (size_t)s * N;
  const int i = lane;
  const bool act = i < NB;
  const int ir = act ? i : 0;
  T d[NB];
  if (lvl <= 1) {
    const double *Dq = v.D + (sb + (N - q)) * NB2;
    load_to_t<T, NB>(d, [&](int j) { return j <= ir ? Dq[ir * NB + j] : Dq[j * NB + ir]; });
  } else {
    load_row4<T, NB>(d, v.Dt + (sb + (N - q)) * NB2 + ir * NB);
  }
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
      stage_w<T, NB>(sX, v.Lr + (sb + (N - pl)) * NB2, lane);
      team_bar(bar);
      syrk_row_w<T, NB>(d, sX, ir);
      team_bar(bar);
    }
    if (pr) {
      stage_w<T, NB>(sX, v.Ll + (sb + (N - pr)) * NB2, lane);
      team_bar(bar);
      syrk_row_w<T, NB>(d, sX, ir);
      team_bar(bar);
    }
  }
  if (!elim) {
    if (act) store_row4<T, NB>(v.Dt + (sb + (N - q)) * NB2 + i * NB, d);
    return;
  }
  const int hh = 1 << lvl;
  const bool hasA = q > hh;
  const int a = q - hh;
  T rinv = T(1);
  const int fail = chol_rows_w<T, NB>(d, rinv, i, sCol, sPiv, bar);
  if (i == 0 && fail) report_not_spd(v.status, s, N + 1 - q);
  if (act) {
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      if (j > i) d[j] = T(0);
      sL[j * LD + i] = d[j];   // by columns: sL[j][k] = L_kj
    }
    store_row4<T, NB>(v.Ld + (sb + (N - q)) * NB2 + i * NB, d);
    sCol[i] = rinv;   // inverse diagonal (column buffers are free now)
    v.invd[(sb + (N - q)) * NB + i] = rinv;
  }
  team_bar(bar);
  // left coupling: L_{a,q} = M_{a,q} L^{-T}, staged for the fill
  if (hasA) {
    T av[NB];
    if (lvl == 0) {
      const double *Ea = v.E + ((size_t)s * (N - 1) + (N - q)) * NB2 + ir * NB;
      load_to_t<T, NB>(av, [&](int k) { return Ea[k]; });
    } else {
      const T *Wa = v.W + (sb + (N - a)) * NB2;
#pragma unroll
      for (int k = 0; k < NB; ++k) av[k] = Wa[k * NB + ir];
    }
    trsm_row_w<T, NB>(av, sL, sCol);
    if (act) {
      store_row4<T, NB>(v.Ll + (sb + (N - q)) * NB2 + i * NB, av);
      float4 *x4 = reinterpret_cast<float4 *>(sX + i * LD);
#pragma unroll
      for (int g = 0; g < NB / 4; ++g) x4[g] = make_float4(av[4 * g], av[4 * g + 1], av[4 * g + 2], av[4 * g + 3]);
    }
  } else if (act) {
    float4 *La = reinterpret_cast<float4 *>(v.Ll + (sb + (N - q)) * NB2 + i * NB);
#pragma unroll
    for (int g = 0; g < NB / 4; ++g) La[g] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  // right coupling: L_{b,q} = M_{b,q} L^{-T}
  T b[NB];
  if (lvl == 0 || q == N - 1) {
    const double *Eb = v.E + ((size_t)s * (N - 1) + (N - q - 1)) * NB2;
    load_to_t<T, NB>(b, [&](int k) { return Eb[k * NB + ir]; });
  } else {
    load_row4<T, NB>(b, v.W + (sb + (N - q)) * NB2 + ir * NB);
  }
  trsm_row_w<T, NB>(b, sL, sCol);
  if (act) store_row4<T, NB>(v.Lr + (sb + (N - q)) * NB2 + i * NB, b);
  if (hasA) {
    // fill M_{b,a} = -L_{b,q} L_{a,q}^T (rows of L_{a,q} staged in sX)
    team_bar(bar);
    if (act) {
      T w[NB];
      rowdot_w<T, NB, false>(w, b, sX, T(-1));
      store_row4<T, NB>(v.W + (sb + (N - a)) * NB2 + i * NB, w);
    }
  }
  team_bar(bar);
}

// x_1 of tail s with a wide team. sbuf: x1_rows_w_bytes bytes.
template <typename T, int NB>
__host__ __device__ constexpr size_t x1_rows_w_bytes(int nr) {
  return (size_t)nr * NB * sizeof(double) + (size_t)WCfg<NB>::ELEMS * sizeof(T);
}

template <typename T, int NB>
__device__ __forceinline__ void x1_task_rows_w(const TailView<T> &v, void *sbuf, int lane, int bar, int s) {
  constexpr int NB2 = NB * NB, LD = WCfg<NB>::LD, SM = WCfg<NB>::SM;
  const int N = v.N, nr = v.nr, Lc = v.Lc;
  const size_t sb = (size_t)s * N;
  double *sC = (double *)sbuf;
  T *sX = (T *)(sC + nr * NB), *sL = sX + SM, *sCol = sL + SM, *sPiv = sCol + 2 * NB;
  const int i = lane;
  const bool act = i < NB;
  const int ir = act ? i : 0;
  T d[NB];
  if (Lc <= 1) {
    const double *Dq = v.D + sb * NB2;
    load_to_t<T, NB>(d, [&](int j) { return j <= ir ? Dq[ir * NB + j] : Dq[j * NB + ir]; });
  } else {
    load_row4<T, NB>(d, v.Dt + sb * NB2 + ir * NB);
  }
  if (Lc >= 1) {
    const int m = 1 << (Lc - 1);
    stage_w<T, NB>(sX, v.Lr + (sb + (N - m)) * NB2, lane);
    team_bar(bar);
    syrk_row_w<T, NB>(d, sX, ir);
    team_bar(bar);
  }
  T rinv = T(1);
  const int fail = chol_rows_w<T, NB>(d, rinv, i, sCol, sPiv, bar);
  if (i == 0 && fail) report_not_spd(v.status, s, 1);
  if (act) {
    T z[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      if (j > i) d[j] = T(0);
      sL[j * LD + i] = d[j];   // by columns: sL[j][k] = L_kj
      z[j] = T(0);
    }
    store_row4<T, NB>(v.Ld + sb * NB2 + i * NB, d);
    store_row4<T, NB>(v.Lr + sb * NB2 + i * NB, z);
    store_row4<T, NB>(v.Ll + sb * NB2 + i * NB, z);
    v.invd[sb * NB + i] = rinv;
  }
  team_bar(bar);
  if (act) sCol[i] = rinv;
  for (int e = lane; e < nr * NB; e += 64) sC[e] = v.C[(size_t)s * nr * NB + e];
  team_bar(bar);
  // F = C L^{-T} in FP64, one row of C per lane (column sweep within the row)
  for (int c = lane; c < nr; c += 64) {
    double f[NB];
#pragma unroll
    for (int k = 0; k < NB; ++k) f[k] = sC[c * NB + k];
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      f[j] *= to_d<T>(sCol[j]);
#pragma unroll
      for (int k = j + 1; k < NB; ++k) f[k] = fma(-f[j], to_d<T>(sL[j * LD + k]), f[k]);
    }
#pragma unroll
    for (int k = 0; k < NB; ++k) {
      sC[c * NB + k] = f[k];
      v.F[(size_t)s * nr * NB + c * NB + k] = f[k];
    }
  }
  team_bar(bar);
  double *Us = v.U + (size_t)s * nr * nr;
  for (int e = lane; e < nr * nr; e += 64) {
    const int a = e / nr, b = e - a * nr;
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < NB; ++k) acc = fma(sC[a * NB + k], sC[b * NB + k], acc);
    Us[e] = acc;
  }
}

template <typename T, int NB>
__global__ void __launch_bounds__(128) k_level_rows_w(TailView<T> v, int lvl) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int team = threadIdx.x / 64, lane = threadIdx.x % 64;
  T *sb = (T *)smem_raw + team * WCfg<NB>::ELEMS;
  const int N = v.N, S = v.S;
  const int E = level_elims(N, lvl);
  const int G = lvl == 0 ? 0 : ((N - 1) >> (lvl + 1)) + 1;
  const long g = (long)blockIdx.x * (blockDim.x / 64) + team;
  pdl_wait();
  if (g < (long)S * (E + G)) {
    int s, q;
    bool elim;
    if (g < (long)S * E) {
      s = (int)(g / E);
      q = (2 * (int)(g - (long)s * E) + 1) << lvl;
      elim = true;
    } else {
      const long g2 = g - (long)S * E;
      s = (int)(g2 / G);
      const int j = (int)(g2 - (long)s * G);
      q = j < G - 1 ? (j + 1) << (lvl + 1) : N;
      elim = false;
    }
    factor_task_rows_w<T, NB>(v, sb, lane, 1 + team, s, q, lvl, elim);
  }
  pdl_trigger();
}

template <typename T, int NB>
__global__ void __launch_bounds__(256) k_top_rows_w(TailView<T> v, int lvl0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int team = threadIdx.x / 64, lane = threadIdx.x % 64, teams = blockDim.x / 64;
  T *sb = (T *)smem_raw + team * WCfg<NB>::ELEMS;
  const int N = v.N, s = blockIdx.x;
  pdl_wait();
  for (int lvl = lvl0; lvl < v.Lc; ++lvl) {
    const int E = level_elims(N, lvl);
    const int G = lvl == 0 ? 0 : ((N - 1) >> (lvl + 1)) + 1;
    for (int t = team; t < E + G; t += teams) {
      const bool elim = t < E;
      const int q = elim ? (2 * t + 1) << lvl : (t - E < G - 1 ? (t - E + 1) << (lvl + 1) : N);
      factor_task_rows_w<T, NB>(v, sb, lane, 1 + team, s, q, lvl, elim);
    }
    __syncthreads();
  }
  if (team == 0) x1_task_rows_w<T, NB>(v, smem_raw, lane, 1, s);
  pdl_trigger();
}

template <typename T, int NB>
cudaError_t prepare_rows_w() {
  cudaError_t e = cudaFuncSetAttribute(k_level_rows_w<T, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, 120 * 1024);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_top_rows_w<T, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

template <typename T, int NB>
void launch_tail_rows_w(const TailView<T> &v, cudaStream_t st) {
  const int Tl = top_level(v.N);
  const size_t per = (size_t)WCfg<NB>::ELEMS * sizeof(T);
  for (int l = 0; l < Tl; ++l) {
    const int E = level_elims(v.N, l);
    const int G = l == 0 ? 0 : ((v.N - 1) >> (l + 1)) + 1;
    const long tasks = (long)v.S * (E + G);
    const long blocks = (tasks + 1) / 2;
    launch_pdl(k_level_rows_w<T, NB>, (unsigned)blocks, 128, 2 * per, st, v, l);
  }
  size_t smem = 4 * per;
  const size_t x1b = x1_rows_w_bytes<T, NB>(v.nr);
  if (x1b > smem) smem = x1b;
  launch_pdl(k_top_rows_w<T, NB>, (unsigned)v.S, 256, smem, st, v, Tl);
}

}  // namespace rows
}  // namespace bm
