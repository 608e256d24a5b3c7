// FP64 tail factorization with compile-time block sizes and per-level team
// sizes (Alg. 1, steps 1-3).
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
#include "bm_team.cuh"

namespace bm {
namespace {

template <int NB>
struct TeamSmem {
  static constexpr int doubles = 3 * NB * NB + NB;   // sD, sB, sA, sInv
};

// One task of level lvl: the Schur update of position q gathered from its
// level lvl-1 neighbours and, if q belongs to level lvl, its elimination.
template <int NB, int TEAM>
__device__ __forceinline__ void factor_task(const F64View &v, const Team<TEAM> &tm, double *sD, int s, int q,
                                            int lvl, bool elim) {
  constexpr int NB2 = NB * NB;
  const int N = v.N;
  double *sB = sD + NB2, *sA = sB + NB2, *sInv = sA + NB2;
  const size_t sb = (size_t)s * N;

  team_copy<TEAM, NB2>(tm, sD, (lvl <= 1 ? v.D : v.Dt) + (sb + (N - q)) * NB2);
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
    if (pl) team_syrk_sub<TEAM, NB, double>(tm, sD, sB, pr ? sA : nullptr);
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
    team_copy_t<TEAM, NB, double>(tm, sB, v.E + ((size_t)s * (N - 1) + (N - q - 1)) * NB2);
  else
    team_copy<TEAM, NB2>(tm, sB, v.W + (sb + (N - q)) * NB2);
  if (hasA) {
    if (lvl == 0)
      team_copy<TEAM, NB2>(tm, sA, v.E + ((size_t)s * (N - 1) + (N - q)) * NB2);
    else
      team_copy_t<TEAM, NB, double>(tm, sA, v.W + (sb + (N - a)) * NB2);
  }
  tm.sync();
  const int fail = team_chol<TEAM, NB, double>(tm, sD, sInv);
  if (tm.lane == 0 && fail) report_not_spd(v.status, s, N + 1 - q);
  team_store_lower<TEAM, NB, double>(tm, v.Ld + (sb + (N - q)) * NB2, sD);
  team_trsm_lt<TEAM, NB, double>(tm, sB, hasA ? 2 * NB : NB, sD, sInv);
  team_copy<TEAM, NB2>(tm, v.Lr + (sb + (N - q)) * NB2, sB);
  if (hasA) {
    team_copy<TEAM, NB2>(tm, v.Ll + (sb + (N - q)) * NB2, sA);
    team_gemm_nt_neg<TEAM, NB, double>(tm, v.W + (sb + (N - a)) * NB2, sB, sA);
  } else {
    team_zero<TEAM, NB2>(tm, v.Ll + (sb + (N - q)) * NB2);
  }
  team_copy<TEAM, NB>(tm, v.invd + (sb + (N - q)) * NB, sInv);
  tm.sync();
}

// x_1 of tail s: last update, L_{i,1}, F_{i,1} = C_{i,1} L_{i,1}^{-T}
// (Theorem 1) and U_i = F_{i,1} F_{i,1}^T. sbuf holds 2 NB^2 + max(nr NB,
// NB^2) + NB doubles.
template <int NB, int TEAM>
__device__ __forceinline__ void x1_task(const F64View &v, const Team<TEAM> &tm, double *sbuf, int s) {
  constexpr int NB2 = NB * NB;
  const int N = v.N, nr = v.nr, Lc = v.Lc;
  double *sD = sbuf, *sB = sD + NB2, *sC = sB + NB2;
  double *sInv = sC + (nr * NB > NB2 ? nr * NB : NB2);
  const size_t sb = (size_t)s * N;
  team_copy<TEAM, NB2>(tm, sD, (Lc <= 1 ? v.D : v.Dt) + sb * NB2);
  if (Lc >= 1) {
    const int m = 1 << (Lc - 1);
    team_copy<TEAM, NB2>(tm, sB, v.Lr + (sb + (N - m)) * NB2);
  }
  for (int i = tm.lane; i < nr * NB; i += TEAM) sC[i] = v.C[(size_t)s * nr * NB + i];
  tm.sync();
  if (Lc >= 1) {
    team_syrk_sub<TEAM, NB, double>(tm, sD, sB, nullptr);
    tm.sync();
  }
  const int fail = team_chol<TEAM, NB, double>(tm, sD, sInv);
  if (tm.lane == 0 && fail) report_not_spd(v.status, s, 1);
  team_store_lower<TEAM, NB, double>(tm, v.Ld + sb * NB2, sD);
  team_zero<TEAM, NB2>(tm, v.Ll + sb * NB2);
  team_zero<TEAM, NB2>(tm, v.Lr + sb * NB2);
  team_copy<TEAM, NB>(tm, v.invd + sb * NB, sInv);
  team_trsm_lt<TEAM, NB, double>(tm, sC, nr, sD, sInv);
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

template <int NB>
__host__ __device__ constexpr int x1_doubles(int nr) {
  return 2 * NB * NB + (nr * NB > NB * NB ? nr * NB : NB * NB) + NB;
}

// Grid-wide level: tasks of all tails, eliminated positions first.
template <int NB, int TEAM>
__global__ void __launch_bounds__(256) k_factor_level_team(F64View v, int lvl) {
  extern __shared__ double smem[];
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
    factor_task<NB, TEAM>(v, tm, smem + tm.id * TeamSmem<NB>::doubles, s, q, lvl, elim);
  }
  pdl_trigger();
}

// Top levels lvl0..Lc-1 and x_1 of one tail per CTA.
template <int NB, int TEAM>
__global__ void __launch_bounds__(512) k_factor_top(F64View v, int lvl0) {
  extern __shared__ double smem[];
  const Team<TEAM> tm;
  const int tpc = blockDim.x / TEAM;
  const int N = v.N, s = blockIdx.x;
  constexpr int per = TeamSmem<NB>::doubles;
  pdl_wait();
  for (int lvl = lvl0; lvl < v.Lc; ++lvl) {
    const int E = level_elims(N, lvl);
    const int G = lvl == 0 ? 0 : ((N - 1) >> (lvl + 1)) + 1;
    for (int t = tm.id; t < E + G; t += tpc) {
      const bool elim = t < E;
      const int q = elim ? (2 * t + 1) << lvl : (t - E < G - 1 ? (t - E + 1) << (lvl + 1) : N);
      factor_task<NB, TEAM>(v, tm, smem + tm.id * per, s, q, lvl, elim);
    }
    __syncthreads();
  }
  if (tm.id == 0) x1_task<NB, TEAM>(v, tm, smem, s);
  pdl_trigger();
}

int pick_team(long tasks, int nb) {
  // about two warps' worth of lanes per SM sub-partition (152 SMs x 4)
  const long want = 38912 / (tasks > 0 ? tasks : 1);
  int t = 8;
  while (t < want && t < 128) t <<= 1;
  const int tmin = nb <= 16 ? 8 : nb <= 32 ? 16 : 32;
  return t < tmin ? tmin : t;
}

template <typename... KArgs, typename... Args>
void launch_pdl(void (*kern)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t st,
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
  cudaLaunchKernelEx(&cfg, kern, args...);
}

template <int NB, int TEAM>
void launch_level(const F64View &v, int lvl, long tasks, cudaStream_t st) {
  const size_t per = TeamSmem<NB>::doubles * sizeof(double);
  int tpc = TEAM >= 128 ? 1 : 128 / TEAM;
  while (tpc > 1 && per * tpc > 200 * 1024) tpc >>= 1;
  const long blocks = (tasks + tpc - 1) / tpc;
  launch_pdl(k_factor_level_team<NB, TEAM>, (unsigned)blocks, TEAM * tpc, per * tpc, st, v, lvl);
}

template <int NB, int TEAM>
void launch_top(const F64View &v, int lvl0, cudaStream_t st) {
  const size_t per = TeamSmem<NB>::doubles * sizeof(double);
  const size_t x1b = x1_doubles<NB>(v.nr) * sizeof(double);
  int tpc = TEAM >= 128 ? 4 : 512 / TEAM > 4 ? 4 : 512 / TEAM;
  while (tpc > 1 && per * tpc > 200 * 1024) tpc >>= 1;
  const size_t smem = per * tpc > x1b ? per * tpc : x1b;
  launch_pdl(k_factor_top<NB, TEAM>, (unsigned)v.S, TEAM * tpc, smem, st, v, lvl0);
}

template <int NB, int TEAM>
cudaError_t prepare_one() {
  cudaError_t e = cudaFuncSetAttribute(k_factor_level_team<NB, TEAM>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_factor_top<NB, TEAM>, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
}

template <int NB>
cudaError_t prepare_nb() {
  cudaError_t e;
  if ((e = prepare_one<NB, 8>()) != cudaSuccess) return e;
  if ((e = prepare_one<NB, 16>()) != cudaSuccess) return e;
  if ((e = prepare_one<NB, 32>()) != cudaSuccess) return e;
  if ((e = prepare_one<NB, 64>()) != cudaSuccess) return e;
  return prepare_one<NB, 128>();
}

// First level handled by the per-tail top kernel: the first one with at
// most four positions per tail.
int top_level(int N) {
  const int Lc = chain_levels(N);
  for (int l = 0; l < Lc; ++l) {
    const int tasks = l == 0 ? N / 2 : ((N - 1) >> l) + 1;
    if (tasks <= 4) return l;
  }
  return Lc;
}

template <int NB>
void launch_tail_nb(const F64View &v, cudaStream_t st) {
  const int T = top_level(v.N);
  for (int l = 0; l < T; ++l) {
    const int E = level_elims(v.N, l);
    const int G = l == 0 ? 0 : ((v.N - 1) >> (l + 1)) + 1;
    const long tasks = (long)v.S * (E + G);
    switch (pick_team(tasks, NB)) {
      case 8: launch_level<NB, 8>(v, l, tasks, st); break;
      case 16: launch_level<NB, 16>(v, l, tasks, st); break;
      case 32: launch_level<NB, 32>(v, l, tasks, st); break;
      case 64: launch_level<NB, 64>(v, l, tasks, st); break;
      default: launch_level<NB, 128>(v, l, tasks, st); break;
    }
  }
  if (NB <= 16)
    launch_top<NB, 64>(v, T, st);
  else
    launch_top<NB, 128>(v, T, st);
}

}  // namespace

#define BM_TEAM_NB_LIST(X) X(2) X(3) X(4) X(6) X(8) X(12) X(16) X(24) X(32) X(48)

bool f64_team_supported(int nb) {
  switch (nb) {
#define X(n) case n:
    BM_TEAM_NB_LIST(X)
#undef X
    return true;
  }
  return false;
}

cudaError_t f64_team_prepare() {
  cudaError_t e = cudaSuccess;
#define X(n) \
  if (e == cudaSuccess) e = prepare_nb<n>();
  BM_TEAM_NB_LIST(X)
#undef X
  return e;
}

// Number of kernels the tail part of one factor launches.
int f64_team_tail_launches(int N) { return top_level(N) + 1; }

// Tail levels and x_1 of the factor (the root step stays in bm_fp64.cu).
void f64_team_launch_tail(const F64View &v, cudaStream_t st) {
  switch (v.nb) {
#define X(n)                    \
  case n:                       \
    launch_tail_nb<n>(v, st);   \
    break;
    BM_TEAM_NB_LIST(X)
#undef X
  }
}

}  // namespace bm
