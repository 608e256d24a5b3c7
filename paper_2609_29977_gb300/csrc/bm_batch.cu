// Batched form: many independent branch-MPC systems of uneven S, N, nb in
// one solver object, mixed precision (FP32 tails, FP64 root, FP64
// refinement) as on the single-system path (bm_mixed.cu).
//
// Factor: ONE persistent launch for the whole batch. The work of every
// system -- the tail positions of each odd-even level of Gamma_{N-1}
// (Sec. II), the x_1 block with the coupling solve and local Schur update
// (Alg. 1 steps 1-3), and the root reduction and root Cholesky (steps 4-5)
// -- is laid out as items in one queue per block size, ordered by level.
// Teams of the persistent CTAs take items in queue order; an item waits
// (bounded spin on acquire loads) until the counter of completed items of
// its tail says that all earlier levels of that tail are done, and a root
// item waits until all x_1 items of its system are done. Items are handed
// out in an order in which every dependency of an item precedes it, and an
// item is only handed to a running team, so the waits always end; a wait
// that exceeds its bound records BM_ERR_TIMEOUT and gives up. A CTA serves
// its home queue first and then the others, so uneven systems balance.
//
// Solve: per refinement step three launches over all tails of all systems
// (one CTA per tail): forward substitution (the last CTA of each system does
// its root step), backward substitution with x += d, and the FP64 residual
// (the last CTA of each system evaluates its backward error and raises its
// converged flag, after which that system's CTAs return at once).
//
// Autotuner: the persistent launch shape (threads per CTA, CTAs per SM) is
// picked by timing candidate shapes on the first factor of a handle; the
// choice is cached per batch signature and GPU in a small JSON file.
#include <cuda_runtime.h>
#include <stdio.h>
#include <sys/stat.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "bm_batch.cuh"
#include "bm_tail_rows.cuh"

namespace bm {
bool tune_cache_lookup(const std::string &key, std::vector<int> &vals);
void tune_cache_store(const std::string &key, const std::vector<int> &vals);

size_t mixed_bytes(int S, int N, int nb, int nr);

namespace {
using namespace mx;

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Lane 0 spins until *cnt >= need, for at most `limit` SM clock cycles;
// a wait that runs out records BM_ERR_TIMEOUT in the system's status, and
// later waits of a system that already timed out give up at once. Every
// lane then performs its own acquire load so the team's later reads see the
// producers' writes.
__device__ __forceinline__ void wait_count(const unsigned *cnt, unsigned need, unsigned long long limit, Status *st,
                                           int lane, unsigned mask) {
  if (lane == 0 && ld_acquire(cnt) < need) {
    const long long t0 = clock64();
    while (ld_acquire(cnt) < need) {
      if (*((volatile int *)&st->code) == (int)BM_ERR_TIMEOUT) break;
      if ((unsigned long long)(clock64() - t0) > limit) {
        atomicCAS(&st->code, 0, (int)BM_ERR_TIMEOUT);
        break;
      }
      __nanosleep(128);
    }
  }
  __syncwarp(mask);
  (void)ld_acquire(cnt);
}

__device__ __forceinline__ void signal_count(unsigned *cnt, int lane, unsigned mask) {
  __syncwarp(mask);
  if (lane == 0) {
    __threadfence();
    atomicAdd(cnt, 1u);
  }
}

__device__ __forceinline__ int tasks_per_tail(int N, int l) { return l == 0 ? N / 2 : ((N - 1) >> l) + 1; }

__device__ __forceinline__ unsigned items_before(int N, int l) {
  unsigned c = 0;
  for (int k = 0; k < l; ++k) c += (unsigned)tasks_per_tail(N, k);
  return c;
}

// Root item: R~ = R - sum_i U_i (fixed order), L_R = chol(R~), in FP64 in
// global memory, by one team.
__device__ void root_item(const BInst &I, const double *R, int lane, int TS, unsigned mask, int bar) {
  auto sync = [&]() {
    if (bar) rows::team_bar(bar); else __syncwarp(mask);
  };
  const int nr = I.nr, S = I.S;
  double *Rt = I.m.Rt, *LR = I.m.LR;
  const double *U = I.m.U;
  for (int e = lane; e < nr * nr; e += TS) {
    const int i = e / nr, j = e - i * nr;
    if (j > i) continue;
    const double v = R[i * nr + j] - root_sum_serial(U, S, nr, i, j);
    Rt[i * nr + j] = v;
    Rt[j * nr + i] = v;
    LR[i * nr + j] = v;
    if (j < i) LR[j * nr + i] = 0.0;
  }
  sync();
  int fail = 0;
  for (int j = 0; j < nr; ++j) {
    sync();
    double d = LR[j * nr + j];
    if (!pivot_ok(d)) {
      if (!fail) fail = j + 1;
      d = 1.0;
    }
    const double r = rsqrt(d);
    sync();
    if (lane == 0) LR[j * nr + j] = d * r;
    for (int i = j + 1 + lane; i < nr; i += TS) LR[i * nr + j] *= r;
    sync();
    for (int e = lane; e < (nr - 1 - j) * (nr - 1 - j); e += TS) {
      const int a = e / (nr - 1 - j), b = e - a * (nr - 1 - j);
      if (b > a) continue;
      const int i = j + 1 + a, k = j + 1 + b;
      LR[i * nr + k] = fma(-LR[i * nr + j], LR[k * nr + j], LR[i * nr + k]);
    }
  }
  sync();
  if (lane == 0 && fail) report_not_spd(I.m.status, -1, 0);
}

template <typename T>
__device__ __forceinline__ TailView<T> tail_view(const BInst &I, const double *D, const double *E, const double *C,
                                                 const double *R) {
  TailView<T> v{};
  v.S = I.S; v.N = I.N; v.nb = I.nb; v.nr = I.nr; v.Lc = I.Lc;
  v.D = D; v.E = E; v.C = C; v.R = R;
  v.Ld = I.m.Ld; v.Ll = I.m.Ll; v.Lr = I.m.Lr; v.Dt = I.m.Dt; v.W = I.m.W; v.invd = I.m.invd;
  v.F = I.m.F; v.U = I.m.U; v.status = I.m.status;
  return v;
}

// Decode item idx of class c into (system, level, tail, position).
__device__ __forceinline__ const BSeg &find_seg(const BClass &c, long idx) {
  int lo = 0, hi = c.nseg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (c.segs[mid].start <= idx) lo = mid; else hi = mid - 1;
  }
  return c.segs[lo];
}

// Worker loop of one team over the queue of class c: register-row tasks,
// one warp or less per task for block sizes <= 32, two warps (named barrier
// per team) for larger blocks.
template <int NB>
__device__ void class_worker(const BClass &c, const BInst *inst, const double *const *Dp, const double *const *Ep,
                             const double *const *Cp, const double *const *Rp, unsigned char *smem,
                             unsigned long long limit) {
  constexpr bool WIDE = NB > 32;
  constexpr int NBn = WIDE ? 32 : NB;        // narrow instantiation (unused when WIDE)
  constexpr int NBw = WIDE ? NB : 48;        // wide instantiation (unused when narrow)
  constexpr int TS = WIDE ? 64 : rows::Cfg<NBn>::TS;
  const int team = threadIdx.x / TS, lane = threadIdx.x % TS;
  const unsigned mask =
      TS >= 32 ? 0xffffffffu : (((1u << (TS & 31)) - 1u) << ((threadIdx.x & 31) / TS * TS));
  const int bar = 1 + team;
  unsigned char *tsm = smem + (size_t)team * c.team_bytes;
  __shared__ unsigned long long s_idx[8];
  auto team_sync = [&]() {
    if (WIDE) rows::team_bar(bar); else __syncwarp(mask);
  };
  while (true) {
    unsigned long long idx = 0;
    if (lane == 0) idx = atomicAdd(c.head, 1ull);
    if (WIDE) {
      if (lane == 0) s_idx[team] = idx;
      rows::team_bar(bar);
      idx = s_idx[team];
      rows::team_bar(bar);
    } else {
      idx = __shfl_sync(mask, idx, (threadIdx.x & 31) & ~(TS - 1));
    }
    if ((long)idx >= c.nitems) break;
    const BSeg sg = find_seg(c, (long)idx);
    const BInst &I = inst[sg.inst];
    const long j = (long)idx - sg.start;
    const double *D = Dp[sg.inst], *E = Ep[sg.inst], *C = Cp[sg.inst], *R = Rp[sg.inst];
    const TailView<float> v = tail_view<float>(I, D, E, C, R);
    const int N = I.N, lvl = sg.level;
    if (lvl < I.Lc) {
      const int Ee = level_elims(N, lvl), G = lvl == 0 ? 0 : ((N - 1) >> (lvl + 1)) + 1;
      int s, q;
      bool elim;
      if (j < (long)I.S * Ee) {
        s = (int)(j / Ee);
        q = (2 * (int)(j - (long)s * Ee) + 1) << lvl;
        elim = true;
      } else {
        const long j2 = j - (long)I.S * Ee;
        s = (int)(j2 / G);
        const int jj = (int)(j2 - (long)s * G);
        q = jj < G - 1 ? (jj + 1) << (lvl + 1) : N;
        elim = false;
      }
      if (lvl > 0) {
        wait_count(&I.tail_done[s], items_before(N, lvl), limit, I.m.status, lane, mask);
        team_sync();
      }
      if (WIDE)
        rows::factor_task_rows_w<float, NBw>(v, (float *)tsm, lane, bar, s, q, lvl, elim);
      else
        rows::factor_task_rows<float, NBn>(v, (float *)tsm, lane, mask, s, q, lvl, elim);
      team_sync();
      signal_count(&I.tail_done[s], lane, mask);
    } else if (lvl == I.Lc) {
      const int s = (int)j;
      if (I.Lc > 0) {
        wait_count(&I.tail_done[s], items_before(N, I.Lc), limit, I.m.status, lane, mask);
        team_sync();
      }
      if (WIDE)
        rows::x1_task_rows_w<float, NBw>(v, tsm, lane, bar, s);
      else
        rows::x1_task_rows<float, NBn>(v, tsm, lane, mask, s);
      team_sync();
      signal_count(I.x1_done, lane, mask);
    } else {
      wait_count(I.x1_done, (unsigned)I.S, limit, I.m.status, lane, mask);
      team_sync();
      root_item(I, R, lane, TS, mask, WIDE ? bar : 0);
    }
    team_sync();
  }
}

// Resets the per-factor counters and status words of every system and
// publishes its inputs for the solves.
__global__ void k_batch_prep(BInst *inst, int ninst, BClass *cls, int ncls, const double *const *Dp,
                             const double *const *Ep, const double *const *Cp, const double *const *Rp) {
  const int b = blockIdx.x;
  if (b < ninst) {
    BInst &I = inst[b];
    for (int s = threadIdx.x; s < I.S; s += blockDim.x) I.tail_done[s] = 0u;
    if (threadIdx.x == 0) {
      *I.x1_done = 0u;
      memset(I.m.status, 0, sizeof(Status));
      for (int k = 0; k < 4; ++k) I.m.tickets[k] = 0u;
      I.m.D = Dp[b];
      I.m.E = Ep[b];
      I.m.C = Cp[b];
      I.m.R = Rp[b];
    }
  }
  if (b == 0)
    for (int c = threadIdx.x; c < ncls; c += blockDim.x) *cls[c].head = 0ull;
}

// The queue of one block-size class (cls[c], block size NB) in its own
// persistent launch: the classes run as parallel branches, each SM mostly
// holding one class's code, instead of one launch whose CTAs visit every
// class (and whose SMs then ran the task bodies of all block sizes at once).
template <int NB>
__global__ void __launch_bounds__(256) k_batch_factor_nb(const BClass *cls, int c, BInst *inst,
                                                         const double *const *Dp, const double *const *Ep,
                                                         const double *const *Cp, const double *const *Rp,
                                                         unsigned long long limit) {
  extern __shared__ __align__(16) unsigned char smem[];
  pdl_wait();
  class_worker<NB>(cls[c], inst, Dp, Ep, Cp, Rp, smem, limit);
}



template <int NB>
int team_bytes_for(int nr) {
  if (NB <= 32) {
    const size_t a = (size_t)rows::Cfg<(NB <= 32 ? NB : 32)>::SM * sizeof(float);
    const size_t b = rows::x1_rows_bytes<float, (NB <= 32 ? NB : 32)>(nr);
    return (int)align_up(a > b ? a : b, 16);
  }
  const size_t a = (size_t)rows::WCfg<(NB > 32 ? NB : 48)>::ELEMS * sizeof(float);
  const size_t b = rows::x1_rows_w_bytes<float, (NB > 32 ? NB : 48)>(nr);
  return (int)align_up(a > b ? a : b, 16);
}

int team_width(int nb) { return nb <= 4 ? 4 : nb <= 8 ? 8 : nb <= 16 ? 16 : nb <= 32 ? 32 : 64; }

int batch_team_bytes(int nb, int nr) {
  switch (nb) {
#define X(n) \
  case n:    \
    return team_bytes_for<n>(nr);
    BM_BATCH_NB_LIST(X)
#undef X
  }
  return 0;
}

bool batch_nb_ok(int nb) {
  switch (nb) {
#define X(n) case n:
    BM_BATCH_NB_LIST(X)
#undef X
    return true;
  }
  return false;
}

// The autotune cache (bm_tune.cu) keeps [threads, ctas_per_sm] per batch signature.
bool cache_lookup(const std::string &key, int *threads, int *cps) {
  std::vector<int> v;
  if (!tune_cache_lookup(key, v) || v.size() != 2) return false;
  *threads = v[0];
  *cps = v[1];
  return true;
}

void cache_store(const std::string &key, int threads, int cps) { tune_cache_store(key, {threads, cps}); }

// One lane waits with the batched factor's bounded wait on a counter that
// nothing increments: the wait must give up after `limit` cycles and leave
// BM_ERR_TIMEOUT in the status word (the test of bm_test_bounded_wait).
__global__ void k_wait_nothing(const unsigned *cnt, unsigned long long limit, Status *st) {
  wait_count(cnt, 1u, limit, st, (int)threadIdx.x, 0xffffffffu);
}

}  // namespace
}  // namespace bm

using namespace bm;

extern "C" bm_status bm_test_bounded_wait(unsigned long long limit_cycles, void *stream) {
  if (limit_cycles == 0 || limit_cycles > (1ull << 33)) return BM_ERR_INVALID_ARG;   // at most a few seconds
  cudaStream_t st = (cudaStream_t)stream;
  void *mem = nullptr;
  if (cudaMallocAsync(&mem, 256, st) != cudaSuccess) {
    cudaGetLastError();
    return BM_ERR_OOM;
  }
  unsigned *cnt = (unsigned *)mem;
  Status *status = (Status *)((char *)mem + 64);
  Status h{};
  bm_status rc = BM_ERR_CUDA;
  if (cudaMemsetAsync(mem, 0, 256, st) == cudaSuccess) {
    k_wait_nothing<<<1, 32, 0, st>>>(cnt, limit_cycles, status);
    if (cudaMemcpyAsync(&h, status, sizeof(Status), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
        cudaStreamSynchronize(st) == cudaSuccess)
      rc = (bm_status)h.code;
  }
  cudaFreeAsync(mem, st);
  cudaStreamSynchronize(st);
  cudaGetLastError();
  return rc;
}

struct bm_batch_s {
  int count = 0;
  std::vector<bm_desc> descs;
  void *pool = nullptr;
  size_t pool_bytes = 0;
  BInst *d_inst = nullptr;
  BClass *d_cls = nullptr;
  BSeg *d_segs = nullptr;
  BTail *d_tails = nullptr;
  unsigned long long *d_heads = nullptr;
  int ncls = 0, ntails = 0, max_refine = 10;
  double tol = 1e-10;
  int smem_per_team_max = 0, min_team_width = 32;
  std::vector<int> cls_nb, cls_team_bytes;
  int threads = 128, ctas_per_sm = 2, sms = 152;
  bool tuned = false, tuned_from_cache = false;
  std::string key;
  cudaStream_t cap = nullptr;
  cudaStream_t cls_st[8] = {};     // one branch per block-size class
  cudaEvent_t ev_fork = nullptr, ev_join[8] = {};
  cudaGraphExec_t gfac = nullptr, gsol = nullptr;
  const void *fkey[4] = {nullptr, nullptr, nullptr, nullptr};
  const void *skey[2] = {nullptr, nullptr};
  Status *status = nullptr;   // [count] (inside the pool)
  IRCtl *ctl = nullptr;       // [count]
};

static size_t per_inst_bytes(const bm_desc &d) {
  return align_up(mixed_bytes(d.S, d.N, d.nb, d.nr), 256) + align_up((size_t)d.S * sizeof(unsigned), 256) + 256 +
         256 /*tickets*/;
}

extern "C" size_t bm_batch_workspace_bytes(const bm_desc *descs, int count) {
  if (!descs || count < 1) return 0;
  size_t t = 0;
  for (int i = 0; i < count; ++i) {
    const bm_desc &d = descs[i];
    if (d.S < 1 || d.N < 1 || d.nr < 1 || d.nr > 64 || d.S > 65535 || !batch_nb_ok(d.nb)) return 0;
    t += per_inst_bytes(d);
  }
  return t + align_up((size_t)count * sizeof(Status), 256);
}

static size_t smem_for(const bm_batch_s *h, int threads) {
  size_t best = 0;
  for (int c = 0; c < h->ncls; ++c) {
    const int tw = team_width(h->cls_nb[c]);
    const size_t need = (size_t)(threads / tw) * h->cls_team_bytes[c];
    best = need > best ? need : best;
  }
  return best;
}

static void launch_class(bm_batch_s *h, int c, const double *const *D, const double *const *E,
                         const double *const *C, const double *const *R, cudaStream_t st, bool pdl) {
  const unsigned grid = (unsigned)(h->sms * h->ctas_per_sm);
  const size_t smem = (size_t)(h->threads / team_width(h->cls_nb[c])) * h->cls_team_bytes[c];
  const unsigned long long limit = 4000000000ull;   // about 2 s of SM clock
  switch (h->cls_nb[c]) {
#define X(n)                                                                                                    \
  case n:                                                                                                       \
    if (pdl)                                                                                                    \
      launch_pdl(k_batch_factor_nb<n>, grid, (unsigned)h->threads, smem, st, (const BClass *)h->d_cls, c,      \
                 h->d_inst, D, E, C, R, limit);                                                                 \
    else                                                                                                        \
      k_batch_factor_nb<n><<<grid, h->threads, smem, st>>>(h->d_cls, c, h->d_inst, D, E, C, R, limit);        \
    break;
    BM_BATCH_NB_LIST(X)
#undef X
  }
}

// prep, then one persistent launch per block-size class; with more than one
// class they run as parallel branches (streams forked from and joined to st).
static void launch_factor(bm_batch_s *h, const double *const *D, const double *const *E, const double *const *C,
                          const double *const *R, cudaStream_t st) {
  k_batch_prep<<<h->count, 128, 0, st>>>(h->d_inst, h->count, h->d_cls, h->ncls, D, E, C, R);
  if (h->ncls == 1) {
    launch_class(h, 0, D, E, C, R, st, true);
    return;
  }
  cudaEventRecord(h->ev_fork, st);
  for (int c = 0; c < h->ncls; ++c) {
    cudaStreamWaitEvent(h->cls_st[c], h->ev_fork, 0);
    launch_class(h, c, D, E, C, R, h->cls_st[c], false);
    cudaEventRecord(h->ev_join[c], h->cls_st[c]);
  }
  for (int c = 0; c < h->ncls; ++c) cudaStreamWaitEvent(st, h->ev_join[c], 0);
}

static void launch_solve(bm_batch_s *h, const double *const *r, double *const *x, cudaStream_t st) {
  batch_launch_reset(h->d_inst, h->count, st);
  for (int it = 0; it <= h->max_refine; ++it)
    batch_launch_solve_iteration(h->d_inst, h->d_tails, h->ntails, r, x, it, h->max_refine, h->tol, st);
}

extern "C" bm_status bm_batch_analyze(const bm_desc *descs, int count, void *stream, bm_batch *out) {
  (void)stream;
  if (!out) return BM_ERR_INVALID_ARG;
  *out = nullptr;
  if (!descs || count < 1) return BM_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i)
    if (descs[i].precision != BM_PREC_FP32_IR) return BM_ERR_INVALID_ARG;
  const size_t bytes = bm_batch_workspace_bytes(descs, count);
  if (!bytes) return BM_ERR_INVALID_ARG;
  if (tail_factor_prepare() != cudaSuccess) {
    cudaGetLastError();
    return BM_ERR_CUDA;
  }
  bm_batch_s *h = new (std::nothrow) bm_batch_s();
  if (!h) return BM_ERR_OOM;
  h->count = count;
  h->descs.assign(descs, descs + count);
  h->max_refine = descs[0].max_refine > 0 ? descs[0].max_refine : 10;
  h->tol = descs[0].tol > 0.0 ? descs[0].tol : 1e-10;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev);
  h->pool_bytes = bytes;
  if (cudaMalloc(&h->pool, bytes) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return BM_ERR_OOM;
  }
  cudaMemset(h->pool, 0, bytes);
  // carve per-system buffers and build the host tables
  std::vector<BInst> inst(count);
  char *p = (char *)h->pool;
  h->status = (Status *)p;
  p += align_up((size_t)count * sizeof(Status), 256);
  int max_nr = 1;
  for (int b = 0; b < count; ++b) {
    const bm_desc &d = descs[b];
    BInst &I = inst[b];
    I.S = d.S; I.N = d.N; I.nb = d.nb; I.nr = d.nr; I.Lc = chain_levels(d.N);
    MixedState &m = I.m;
    memset(&m, 0, sizeof m);
    m.S = d.S; m.N = d.N; m.nb = d.nb; m.nr = d.nr; m.Lc = I.Lc;
    const size_t SN = (size_t)d.S * d.N, b2 = (size_t)d.nb * d.nb, n = SN * d.nb + d.nr;
    char *q = p;
    auto take = [&](size_t nbytes) {
      void *r = q;
      q += align_up(nbytes, 256);
      return r;
    };
    m.Ld = (float *)take(SN * b2 * 4); m.Ll = (float *)take(SN * b2 * 4); m.Lr = (float *)take(SN * b2 * 4);
    m.Dt = (float *)take(SN * b2 * 4); m.W = (float *)take(SN * b2 * 4);
    m.invd = (float *)take(SN * d.nb * 4); m.y = (float *)take(SN * d.nb * 4); m.zt = (float *)take(SN * d.nb * 4);
    m.F = (double *)take((size_t)d.S * d.nr * d.nb * 8); m.U = (double *)take((size_t)d.S * d.nr * d.nr * 8);
    m.LR = (double *)take((size_t)d.nr * d.nr * 8); m.Rt = (double *)take((size_t)d.nr * d.nr * 8);
    m.tb = (double *)take((size_t)d.S * d.nr * 8); m.d0 = (double *)take((size_t)d.nr * 8);
    m.rho = (double *)take(n * 8);
    m.ctl = (IRCtl *)take(sizeof(IRCtl));
    p += align_up(mixed_bytes(d.S, d.N, d.nb, d.nr), 256);
    I.tail_done = (unsigned *)p;
    p += align_up((size_t)d.S * sizeof(unsigned), 256);
    I.x1_done = (unsigned *)p;
    p += 256;
    m.tickets = (unsigned *)p;
    p += 256;
    m.status = h->status + b;
    max_nr = d.nr > max_nr ? d.nr : max_nr;
  }
  // class queues: items ordered by level, then system
  std::vector<int> nbs;
  for (int b = 0; b < count; ++b)
    if (std::find(nbs.begin(), nbs.end(), descs[b].nb) == nbs.end()) nbs.push_back(descs[b].nb);
  std::sort(nbs.begin(), nbs.end());
  std::vector<BSeg> segs;
  std::vector<BClass> cls;
  for (int nb : nbs) {
    BClass c;
    memset(&c, 0, sizeof c);
    c.nb = nb;
    const int first = (int)segs.size();
    long start = 0;
    int cls_max_nr = 1, maxlev = 0;
    for (int b = 0; b < count; ++b)
      if (descs[b].nb == nb) {
        maxlev = std::max(maxlev, inst[b].Lc + 1);
        cls_max_nr = std::max(cls_max_nr, descs[b].nr);
      }
    for (int l = 0; l <= maxlev; ++l)
      for (int b = 0; b < count; ++b) {
        if (descs[b].nb != nb || l > inst[b].Lc + 1) continue;
        const int S = descs[b].S, N = descs[b].N, Lc = inst[b].Lc;
        long cnt;
        if (l < Lc) {
          const int tpt = l == 0 ? N / 2 : ((N - 1) >> l) + 1;
          cnt = (long)S * tpt;
        } else if (l == Lc) {
          cnt = S;
        } else {
          cnt = 1;
        }
        BSeg sg;
        sg.start = start;
        sg.inst = b;
        sg.level = l;
        sg.count = (int)cnt;
        segs.push_back(sg);
        start += cnt;
      }
    c.nseg = (int)segs.size() - first;
    c.nitems = start;
    c.segs = (const BSeg *)(intptr_t)first;   // fixed up after the upload
    c.team_bytes = batch_team_bytes(nb, cls_max_nr);
    cls.push_back(c);
    h->cls_nb.push_back(nb);
    h->cls_team_bytes.push_back(c.team_bytes);
  }
  h->ncls = (int)cls.size();
  std::vector<BTail> tails;
  for (int b = 0; b < count; ++b)
    for (int s = 0; s < descs[b].S; ++s) tails.push_back(BTail{b, s});
  h->ntails = (int)tails.size();
  bool ok = cudaMalloc(&h->d_inst, count * sizeof(BInst)) == cudaSuccess &&
            cudaMalloc(&h->d_cls, cls.size() * sizeof(BClass)) == cudaSuccess &&
            cudaMalloc(&h->d_segs, segs.size() * sizeof(BSeg)) == cudaSuccess &&
            cudaMalloc(&h->d_tails, tails.size() * sizeof(BTail)) == cudaSuccess &&
            cudaMalloc(&h->d_heads, cls.size() * sizeof(unsigned long long)) == cudaSuccess;
  if (ok) {
    for (size_t c = 0; c < cls.size(); ++c) {
      cls[c].segs = h->d_segs + (intptr_t)cls[c].segs;
      cls[c].head = h->d_heads + c;
    }
    ok = cudaMemcpy(h->d_inst, inst.data(), count * sizeof(BInst), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(h->d_cls, cls.data(), cls.size() * sizeof(BClass), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(h->d_segs, segs.data(), segs.size() * sizeof(BSeg), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(h->d_tails, tails.data(), tails.size() * sizeof(BTail), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) == cudaSuccess;
#define X(n)                                                                                              \
  ok = ok && cudaFuncSetAttribute(k_batch_factor_nb<n>, cudaFuncAttributeMaxDynamicSharedMemorySize,       \
                                  200 * 1024) == cudaSuccess;
    BM_BATCH_NB_LIST(X)
#undef X
    for (int c = 0; ok && c < (int)cls.size(); ++c)
      ok = cudaStreamCreateWithFlags(&h->cls_st[c], cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&h->ev_join[c], cudaEventDisableTiming) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    bm_batch_destroy(h);
    return BM_ERR_CUDA;
  }
  // signature of the batch for the autotune cache
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, dev);
  char kb[256];
  long tot_stages = 0;
  for (int b = 0; b < count; ++b) tot_stages += (long)descs[b].S * descs[b].N;
  snprintf(kb, sizeof kb, "%.200s|n=%d|stages~2^%d|nb=", prop.name, count, 63 - __builtin_clzll((unsigned long long)tot_stages | 1));
  h->key = kb;
  for (int nb : nbs) h->key += std::to_string(nb) + ",";
  *out = h;
  return BM_OK;
}

static bool fits(const bm_batch_s *h, int threads) { return smem_for(h, threads) <= 200 * 1024; }

static bm_status autotune(bm_batch_s *h, const double *const *D, const double *const *E, const double *const *C,
                          const double *const *R, cudaStream_t st) {
  int t0 = 0, c0 = 0;
  if (cache_lookup(h->key, &t0, &c0) && fits(h, t0) && c0 >= 1 && c0 <= 8) {
    h->threads = t0;
    h->ctas_per_sm = c0;
    h->tuned = h->tuned_from_cache = true;
    return BM_OK;
  }
  const int cand[][2] = {{128, 1}, {128, 2}, {128, 3}, {128, 4}, {64, 2}, {64, 4}, {64, 6}, {256, 1}};
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  float best = 1e30f;
  int bt = 128, bc = 2;
  for (const auto &c : cand) {
    if (!fits(h, c[0])) continue;
    h->threads = c[0];
    h->ctas_per_sm = c[1];
    launch_factor(h, D, E, C, R, st);   // warm
    float ms[3];
    for (int k = 0; k < 3; ++k) {
      cudaEventRecord(a, st);
      launch_factor(h, D, E, C, R, st);
      cudaEventRecord(b, st);
      cudaEventSynchronize(b);
      cudaEventElapsedTime(&ms[k], a, b);
    }
    std::sort(ms, ms + 3);
    if (ms[1] < best) {
      best = ms[1];
      bt = c[0];
      bc = c[1];
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (cudaGetLastError() != cudaSuccess) return BM_ERR_CUDA;
  h->threads = bt;
  h->ctas_per_sm = bc;
  h->tuned = true;
  cache_store(h->key, bt, bc);
  return BM_OK;
}

template <typename Body>
static bm_status run_graph(bm_batch_s *h, cudaGraphExec_t *slot, const void **key, const void *const *want, int n,
                           cudaStream_t st, Body body) {
  bool match = *slot != nullptr;
  for (int i = 0; i < n && match; ++i) match = key[i] == want[i];
  if (!match) {
    if (*slot) cudaGraphExecDestroy(*slot);
    *slot = nullptr;
    if (cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return BM_ERR_CUDA;
    body(h->cap);
    cudaGraph_t g = nullptr;
    if (cudaStreamEndCapture(h->cap, &g) != cudaSuccess || !g) {
      cudaGetLastError();
      return BM_ERR_CUDA;
    }
    const cudaError_t e = cudaGraphInstantiate(slot, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      cudaGetLastError();
      *slot = nullptr;
      return BM_ERR_CUDA;
    }
    for (int i = 0; i < n; ++i) key[i] = want[i];
  }
  return cudaGraphLaunch(*slot, st) == cudaSuccess ? BM_OK : BM_ERR_CUDA;
}

extern "C" bm_status bm_batch_factor(bm_batch h, const double *const *D, const double *const *E,
                                     const double *const *C, const double *const *R, void *stream) {
  if (!h || !D || !E || !C || !R) return BM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (!h->tuned) {
    const bm_status s = autotune(h, D, E, C, R, st);
    if (s != BM_OK) return s;
  }
  const void *want[4] = {D, E, C, R};
  return run_graph(h, &h->gfac, h->fkey, want, 4, st,
                   [&](cudaStream_t cs) { launch_factor(h, D, E, C, R, cs); });
}

extern "C" bm_status bm_batch_solve(bm_batch h, const double *const *r, double *const *x, void *stream) {
  if (!h || !r || !x) return BM_ERR_INVALID_ARG;
  if (!h->tuned) return BM_ERR_NOT_FACTORED;
  const void *want[2] = {r, x};
  return run_graph(h, &h->gsol, h->skey, want, 2, (cudaStream_t)stream,
                   [&](cudaStream_t cs) { launch_solve(h, r, x, cs); });
}

extern "C" bm_status bm_batch_query(bm_batch h, void *stream, bm_info *infos) {
  if (!h) return BM_ERR_INVALID_ARG;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
    cudaGetLastError();
    return BM_ERR_CUDA;
  }
  std::vector<Status> st(h->count);
  if (cudaMemcpy(st.data(), h->status, h->count * sizeof(Status), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return BM_ERR_CUDA;
  }
  bm_status first = BM_OK;
  for (int b = 0; b < h->count; ++b) {
    if (infos) {
      infos[b].status = st[b].code;
      infos[b].fail_scenario = st[b].code == BM_ERR_NOT_SPD ? st[b].scenario : 0;
      infos[b].fail_stage = st[b].code == BM_ERR_NOT_SPD ? st[b].stage : 0;
      infos[b].iters = st[b].iters;
      infos[b].backward_error = st[b].eta;
      infos[b].coupling_refined = 0;
      infos[b].residual_float_float = 0;
      infos[b].host_pipelined = 0;
    }
    if (first == BM_OK && st[b].code != 0) first = (bm_status)st[b].code;
  }
  return first;
}

extern "C" bm_status bm_batch_schedule(bm_batch h, int *threads_per_cta, int *ctas_per_sm, int *from_cache) {
  if (!h) return BM_ERR_INVALID_ARG;
  if (threads_per_cta) *threads_per_cta = h->threads;
  if (ctas_per_sm) *ctas_per_sm = h->ctas_per_sm;
  if (from_cache) *from_cache = h->tuned_from_cache ? 1 : 0;
  return h->tuned ? BM_OK : BM_ERR_NOT_FACTORED;
}

extern "C" void bm_batch_destroy(bm_batch h) {
  if (!h) return;
  cudaDeviceSynchronize();
  if (h->gfac) cudaGraphExecDestroy(h->gfac);
  if (h->gsol) cudaGraphExecDestroy(h->gsol);
  if (h->cap) cudaStreamDestroy(h->cap);
  for (int c = 0; c < 8; ++c) {
    if (h->cls_st[c]) cudaStreamDestroy(h->cls_st[c]);
    if (h->ev_join[c]) cudaEventDestroy(h->ev_join[c]);
  }
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  cudaFree(h->d_inst);
  cudaFree(h->d_cls);
  cudaFree(h->d_segs);
  cudaFree(h->d_tails);
  cudaFree(h->d_heads);
  cudaFree(h->pool);
  cudaGetLastError();
  delete h;
}
