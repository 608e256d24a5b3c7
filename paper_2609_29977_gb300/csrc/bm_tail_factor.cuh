// Tail factorization with compile-time block sizes and per-level team sizes
// (Alg. 1, steps 1-3), for the FP64 path (T = double) and the FP32 tails of
// the mixed-precision path (T = float: the FP64 inputs are rounded to
// nearest on load; the coupling solve and the local Schur update stay FP64).
//
// Same level schedule as the generic kernels in bm_fp64.cu (odd-even levels
// of Gamma_{N-1}, Sec. II), organised for GB300:
//  * wide levels (many positions per tail) run as grid-wide launches whose
//    tasks are flattened over all tails, eliminated positions first and
//    update-only positions after them, each task run by a team of TEAM
//    threads sized from the task count: small teams (several per warp) when a
//    level has thousands of tasks, so that the pivot steps of several tasks
//    share a warp instruction and every lane of the FP64 pipe is busy;
//  * the top levels (at most four positions per tail) and x_1 run in one
//    launch with one CTA per tail, the levels separated by __syncthreads,
//    because there the cost is the dependent chain of each level, not the
//    flops, and a kernel boundary per level would add to it;
//  * launches are chained with programmatic dependent launch.
//
// The explicit instantiations live in bm_tail_inst_*.cu so that they compile
// in parallel; bm_tail_factor.cu dispatches on the block size.
#pragma once

#include "bm_root.cuh"
#include "bm_team.cuh"

namespace bm {
namespace tail {

template <typename T, int NB>
struct TeamSmem {
  static constexpr int elems = 3 * NB * NB + NB;   // sD, sB, sA, sInv
  static constexpr size_t bytes = elems * sizeof(T);
};

// Input blocks (FP64 in memory) into shared memory of type T.
template <int TEAM, int N, typename T>
__device__ __forceinline__ void team_load(const Team<TEAM> &tm, T *__restrict__ dst, const double *__restrict__ src) {
#pragma unroll
  for (int i = tm.lane; i < N; i += TEAM) dst[i] = to_t<T>(src[i]);
}
template <int TEAM, int NB, typename T>
__device__ __forceinline__ void team_load_t(const Team<TEAM> &tm, T *__restrict__ dst, const double *__restrict__ src) {
#pragma unroll
  for (int e = tm.lane; e < NB * NB; e += TEAM) {
    const int i = e / NB, j = e - i * NB;
    dst[j * NB + i] = to_t<T>(src[e]);
  }
}

// One task of level lvl: the Schur update of position q gathered from its
// level lvl-1 neighbours and, if q belongs to level lvl, its elimination.
template <typename T, int NB, int TEAM>
__device__ __forceinline__ void factor_task(const TailView<T> &v, const Team<TEAM> &tm, T *sD, int s, int q,
                                            int lvl, bool elim) {
  constexpr int NB2 = NB * NB;
  const int N = v.N;
  T *sB = sD + NB2, *sA = sB + NB2, *sInv = sA + NB2;
  const size_t sb = (size_t)s * N;

  if (lvl <= 1)
    team_load<TEAM, NB2, T>(tm, sD, v.D + (sb + (N - q)) * NB2);
  else
    team_copy<TEAM, NB2>(tm, sD, v.Dt + (sb + (N - q)) * NB2);
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
    if (pl) team_copy<TEAM, NB2>(tm, sB, v.Lr + (sb + (N - pl)) * NB2);
    if (pr) team_copy<TEAM, NB2>(tm, sA, v.Ll + (sb + (N - pr)) * NB2);
    tm.sync();
    if (pl) team_syrk_sub<TEAM, NB, T>(tm, sD, sB, pr ? sA : nullptr);
    tm.sync();
  }
  if (!elim) {
    team_copy<TEAM, NB2>(tm, v.Dt + (sb + (N - q)) * NB2, sD);
    tm.sync();
    return;
  }
  // couplings to the right and left neighbours, loaded before the Cholesky
  // so their latency hides behind it: M_{b,q} is the original block at level
  // 0 and for the last chain position (whose right neighbour is always
  // x_1), else the fill left by the previous level; M_{a,q} likewise.
  const int h = 1 << lvl;
  const bool hasA = q > h;
  const int a = q - h;
  if (lvl == 0 || q == N - 1)
    team_load_t<TEAM, NB, T>(tm, sB, v.E + ((size_t)s * (N - 1) + (N - q - 1)) * NB2);
  else
    team_copy<TEAM, NB2>(tm, sB, v.W + (sb + (N - q)) * NB2);
  if (hasA) {
    if (lvl == 0)
      team_load<TEAM, NB2, T>(tm, sA, v.E + ((size_t)s * (N - 1) + (N - q)) * NB2);
    else
      team_copy_t<TEAM, NB, T>(tm, sA, v.W + (sb + (N - a)) * NB2);
  }
  tm.sync();
  const int fail = team_chol<TEAM, NB, T>(tm, sD, sInv);
  if (tm.lane == 0 && fail) report_not_spd(v.status, v.s0 + s, N + 1 - q);
  team_store_factor<TEAM, NB, T>(tm, v.Ld + (sb + (N - q)) * NB2, sD, sInv);
  team_trsm_lt<TEAM, NB, T>(tm, sB, hasA ? 2 * NB : NB, sD, sInv);
  team_copy<TEAM, NB2>(tm, v.Lr + (sb + (N - q)) * NB2, sB);
  if (hasA) {
    team_copy<TEAM, NB2>(tm, v.Ll + (sb + (N - q)) * NB2, sA);
    team_gemm_nt_neg<TEAM, NB, T>(tm, v.W + (sb + (N - a)) * NB2, sB, sA);
  } else {
    team_zero<TEAM, NB2>(tm, v.Ll + (sb + (N - q)) * NB2);
  }
  team_copy<TEAM, NB>(tm, v.invd + (sb + (N - q)) * NB, sInv);
  tm.sync();
}

// x_1 of tail s: last update and L_{i,1} (in T), then in FP64 the coupling
// solve F_{i,1} = C_{i,1} L_{i,1}^{-T} (Theorem 1) and the local Schur update
// U_i = F_{i,1} F_{i,1}^T. sbuf holds x1_bytes<T, NB>(nr) bytes.
template <typename T, int NB>
__host__ __device__ constexpr size_t x1_bytes(int nr) {
  return (size_t)nr * NB * sizeof(double) + (2 * NB * NB + NB) * sizeof(T);
}

template <typename T, int NB, int TEAM>
__device__ __forceinline__ void x1_task(const TailView<T> &v, const Team<TEAM> &tm, void *sbuf, int s) {
  constexpr int NB2 = NB * NB;
  const int N = v.N, nr = v.nr, Lc = v.Lc;
  double *sC = (double *)sbuf;
  T *sD = (T *)(sC + nr * NB), *sB = sD + NB2, *sInv = sB + NB2;
  const size_t sb = (size_t)s * N;
  if (Lc <= 1)
    team_load<TEAM, NB2, T>(tm, sD, v.D + sb * NB2);
  else
    team_copy<TEAM, NB2>(tm, sD, v.Dt + sb * NB2);
  if (Lc >= 1) {
    const int m = 1 << (Lc - 1);
    team_copy<TEAM, NB2>(tm, sB, v.Lr + (sb + (N - m)) * NB2);
  }
  for (int i = tm.lane; i < nr * NB; i += TEAM) sC[i] = v.C[(size_t)s * nr * NB + i];
  tm.sync();
  if (Lc >= 1) {
    team_syrk_sub<TEAM, NB, T>(tm, sD, sB, nullptr);
    tm.sync();
  }
  const int fail = team_chol<TEAM, NB, T>(tm, sD, sInv);
  if (tm.lane == 0 && fail) report_not_spd(v.status, v.s0 + s, 1);
  team_store_factor<TEAM, NB, T>(tm, v.Ld + sb * NB2, sD, sInv);
  team_zero<TEAM, NB2>(tm, v.Ll + sb * NB2);
  team_zero<TEAM, NB2>(tm, v.Lr + sb * NB2);
  team_copy<TEAM, NB>(tm, v.invd + sb * NB, sInv);
  // F = C L^{-T} in FP64: column sweep over the widened factor
#pragma unroll 1
  for (int j = 0; j < NB; ++j) {
    const double r = (double)sInv[j];
    for (int row = tm.lane; row < nr; row += TEAM) sC[row * NB + j] *= r;
    tm.sync();
    const int cols = NB - 1 - j, ne = nr * cols;
    for (int e = tm.lane; e < ne; e += TEAM) {
      const int row = e / cols, k = j + 1 + (e - row * cols);
      sC[row * NB + k] = fma(-sC[row * NB + j], (double)sD[k * NB + j], sC[row * NB + k]);
    }
    tm.sync();
  }
  for (int i = tm.lane; i < nr * NB; i += TEAM) v.F[(size_t)s * nr * NB + i] = sC[i];
  double *Us = v.U + (size_t)s * nr * nr;
  for (int e = tm.lane; e < nr * nr; e += TEAM) {
    const int i = e / nr, j = e - i * nr;
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < NB; ++k) acc = fma(sC[i * NB + k], sC[j * NB + k], acc);
    Us[e] = acc;
  }
}

// Grid-wide level: tasks of all tails, eliminated positions first.
template <typename T, int NB, int TEAM>
__global__ void __launch_bounds__(256) k_factor_level_team(TailView<T> v, int lvl) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *smem = (T *)smem_raw;
  const Team<TEAM> tm;
  const int tpc = blockDim.x / TEAM;
  const int N = v.N, S = v.S;
  const int E = level_elims(N, lvl);
  const int G = lvl == 0 ? 0 : ((N - 1) >> (lvl + 1)) + 1;
  const long g = (long)blockIdx.x * tpc + tm.id;
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
    factor_task<T, NB, TEAM>(v, tm, smem + tm.id * TeamSmem<T, NB>::elems, s, q, lvl, elim);
  }
  pdl_trigger();
}

// Top levels lvl0..Lc-1 and x_1 of one tail per CTA.
template <typename T, int NB, int TEAM>
__global__ void __launch_bounds__(512) k_factor_top(TailView<T> v, int lvl0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *smem = (T *)smem_raw;
  const Team<TEAM> tm;
  const int tpc = blockDim.x / TEAM;
  const int N = v.N, s = blockIdx.x;
  constexpr int per = TeamSmem<T, NB>::elems;
  pdl_wait();
  for (int lvl = lvl0; lvl < v.Lc; ++lvl) {
    const int E = level_elims(N, lvl);
    const int G = lvl == 0 ? 0 : ((N - 1) >> (lvl + 1)) + 1;
    for (int t = tm.id; t < E + G; t += tpc) {
      const bool elim = t < E;
      const int q = elim ? (2 * t + 1) << lvl : (t - E < G - 1 ? (t - E + 1) << (lvl + 1) : N);
      factor_task<T, NB, TEAM>(v, tm, smem + tm.id * per, s, q, lvl, elim);
    }
    __syncthreads();
  }
  if (tm.id == 0) x1_task<T, NB, TEAM>(v, tm, smem_raw, s);
  if constexpr (sizeof(T) == sizeof(double)) {
    if (v.LR) {
      // the last tail to finish its U_i does the root step (Alg. 1 steps 4-5)
      __shared__ int last;
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) last = atomicAdd(&v.tickets[0], 1u) == gridDim.x - 1;
      __syncthreads();
      if (last) {
        __threadfence();
        root_reduce_chol(v.U, v.R, v.S, v.nr, v.Rt, v.LR, v.status, (double *)smem_raw);
        if (threadIdx.x == 0) v.tickets[0] = 0u;
      }
    }
  }
  pdl_trigger();
}

// Team sizes compiled for each block size, and the team of the top kernel.
constexpr int team_min(int nb) { return nb <= 16 ? 8 : nb <= 32 ? 16 : 32; }
constexpr int team_max(int nb) { return nb <= 4 ? 32 : nb <= 16 ? 64 : 128; }
constexpr int team_top(int nb) { return nb <= 8 ? 32 : nb <= 16 ? 64 : 128; }

inline int pick_team(long tasks, int nb) {
  // about two warps' worth of lanes per SM sub-partition (152 SMs x 4)
  const long want = 38912 / (tasks > 0 ? tasks : 1);
  int t = 8;
  while (t < want && t < 128) t <<= 1;
  const int tmin = team_min(nb), tmax = team_max(nb);
  return t < tmin ? tmin : t > tmax ? tmax : t;
}

template <typename T, int NB, int TEAM>
void launch_level(const TailView<T> &v, int lvl, long tasks, cudaStream_t st) {
  const size_t per = TeamSmem<T, NB>::bytes;
  // CTAs of 128 threads, or of 256 when the level has enough tasks to give
  // every SM four such CTAs: the SM then keeps twice the teams resident
  // (measured on the mixed workload's FP64 factor: 6703 -> 6296 us; on the
  // medium workload's smaller levels the larger CTAs leave SMs idle)
  int tpc = TEAM >= 128 ? 1 : 128 / TEAM;
  if (TEAM < 256 && tasks * TEAM >= 256L * 4 * 152) tpc = 256 / TEAM;
  while (tpc > 1 && per * tpc > 200 * 1024) tpc >>= 1;
  const long blocks = (tasks + tpc - 1) / tpc;
  launch_pdl(k_factor_level_team<T, NB, TEAM>, (unsigned)blocks, TEAM * tpc, per * tpc, st, v, lvl);
}

template <typename T, int NB, int TEAM>
void launch_top(const TailView<T> &v, int lvl0, cudaStream_t st) {
  const size_t per = TeamSmem<T, NB>::bytes;
  const size_t x1b = x1_bytes<T, NB>(v.nr);
  int tpc = TEAM >= 128 ? 4 : 512 / TEAM > 4 ? 4 : 512 / TEAM;
  while (tpc > 1 && per * tpc > 200 * 1024) tpc >>= 1;
  size_t smem = per * tpc > x1b ? per * tpc : x1b;
  const size_t rootb = ((size_t)v.nr * v.nr + v.nr) * sizeof(double);
  if (v.LR && rootb > smem) smem = rootb;
  launch_pdl(k_factor_top<T, NB, TEAM>, (unsigned)v.S, TEAM * tpc, smem, st, v, lvl0);
}

template <typename T, int NB, int TEAM>
cudaError_t prepare_one() {
  cudaError_t e = cudaFuncSetAttribute(k_factor_level_team<T, NB, TEAM>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_factor_top<T, NB, TEAM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              210 * 1024);
}

template <typename T, int NB, int TEAM>
cudaError_t prepare_if_compiled() {
  if (TEAM < team_min(NB) || TEAM > team_max(NB)) return cudaSuccess;
  return prepare_one<T, NB, (TEAM < team_min(NB) ? team_min(NB) : TEAM > team_max(NB) ? team_max(NB) : TEAM)>();
}

template <typename T, int NB>
cudaError_t prepare_nb() {
  cudaError_t e;
  if ((e = prepare_if_compiled<T, NB, 8>()) != cudaSuccess) return e;
  if ((e = prepare_if_compiled<T, NB, 16>()) != cudaSuccess) return e;
  if ((e = prepare_if_compiled<T, NB, 32>()) != cudaSuccess) return e;
  if ((e = prepare_if_compiled<T, NB, 64>()) != cudaSuccess) return e;
  return prepare_if_compiled<T, NB, 128>();
}

// Launch the level kernel with a team size that is compiled for NB.
template <typename T, int NB, int TEAM>
void launch_level_clamped(const TailView<T> &v, int lvl, long tasks, cudaStream_t st) {
  constexpr int t = TEAM < team_min(NB) ? team_min(NB) : TEAM > team_max(NB) ? team_max(NB) : TEAM;
  launch_level<T, NB, t>(v, lvl, tasks, st);
}

// Grid-wide levels [lo, min(hi, top)) of the tails in v and, if top, the
// per-tail top kernel. With ev, ev[l] is recorded before level l and ev[top+1]
// after the top kernel.
template <typename T, int NB>
void launch_tail_range(const TailView<T> &v, cudaStream_t st, const TailSched *sc, int lo, int hi, bool top,
                       cudaEvent_t *ev) {
  const int Tl = sc ? sc->top : top_level(v.N);
  if (ev) cudaEventRecord(ev[0], st);
  for (int l = lo; l < Tl && l < hi; ++l) {
    const int E = level_elims(v.N, l);
    const int G = l == 0 ? 0 : ((v.N - 1) >> (l + 1)) + 1;
    const long tasks = (long)v.S * (E + G);
    switch (sc ? sc->team[l] : pick_team(tasks, NB)) {
      case 8: launch_level_clamped<T, NB, 8>(v, l, tasks, st); break;
      case 16: launch_level_clamped<T, NB, 16>(v, l, tasks, st); break;
      case 32: launch_level_clamped<T, NB, 32>(v, l, tasks, st); break;
      case 64: launch_level_clamped<T, NB, 64>(v, l, tasks, st); break;
      default: launch_level_clamped<T, NB, 128>(v, l, tasks, st); break;
    }
    if (ev) cudaEventRecord(ev[l + 1], st);
  }
  if (!top) return;
  launch_top<T, NB, team_top(NB)>(v, Tl, st);
  if (ev) cudaEventRecord(ev[Tl + 1], st);
}

template <typename T, int NB>
void launch_tail_nb(const TailView<T> &v, cudaStream_t st, const TailSched *sc, cudaEvent_t *ev) {
  launch_tail_range<T, NB>(v, st, sc, 0, 1 << 30, true, ev);
}

}  // namespace tail
}  // namespace bm
