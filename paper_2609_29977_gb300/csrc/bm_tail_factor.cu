// Dispatch of the tail factorization on the block size (Alg. 1, steps 1-3).
// The kernels are defined in bm_tail_factor.cuh and instantiated in
// bm_tail_inst_*.cu.
#include <mutex>

#include "bm_tail_factor.cuh"
#include "bm_tail_rows.cuh"

namespace bm {
namespace tail {
#define X(n)                                                                                               \
  extern template void launch_tail_nb<double, n>(const TailView<double> &, cudaStream_t, const TailSched *, \
                                                 cudaEvent_t *);                                           \
  extern template void launch_tail_nb<float, n>(const TailView<float> &, cudaStream_t, const TailSched *,   \
                                                cudaEvent_t *);                                            \
  extern template void launch_tail_range<double, n>(const TailView<double> &, cudaStream_t, const TailSched *, \
                                                    int, int, bool, cudaEvent_t *);                            \
  extern template cudaError_t prepare_nb<double, n>();                              \
  extern template cudaError_t prepare_nb<float, n>();
BM_TAIL_NB_LIST(X)
#undef X
}  // namespace tail
namespace rows {
#define X(n)                                                                                  \
  extern template void launch_tail_rows<float, n>(const TailView<float> &, cudaStream_t); \
  extern template cudaError_t prepare_rows<float, n>();
BM_ROWS_NB_LIST(X)
#undef X
extern template void launch_tail_rows_w<float, 48>(const TailView<float> &, cudaStream_t);
extern template cudaError_t prepare_rows_w<float, 48>();
}  // namespace rows

bool tail_nb_supported(int nb) {
  switch (nb) {
#define X(n) case n:
    BM_TAIL_NB_LIST(X)
#undef X
    return true;
  }
  return false;
}

cudaError_t tail_factor_prepare() {
  static std::mutex mu;
  static bool done[64] = {false};
  std::lock_guard<std::mutex> lock(mu);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return cudaErrorUnknown;
  if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
  cudaError_t e = cudaSuccess;
#define X(n)                                                   \
  if (e == cudaSuccess) e = tail::prepare_nb<double, n>();     \
  if (e == cudaSuccess) e = tail::prepare_nb<float, n>();
  BM_TAIL_NB_LIST(X)
#undef X
#define X(n) \
  if (e == cudaSuccess) e = rows::prepare_rows<float, n>();
  BM_ROWS_NB_LIST(X)
#undef X
  if (e == cudaSuccess) e = rows::prepare_rows_w<float, 48>();
  if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
  return e;
}

// Tail levels and x_1 of the factor (the root step is launched separately).
// FP32 tails use the register-row kernels (two-warp teams for nb = 48).
template <typename T>
void tail_factor_launch(const TailView<T> &v, cudaStream_t st, const TailSched *sc, cudaEvent_t *ev) {
  if (sizeof(T) == 4) {
    switch (v.nb) {
#define X(n)                                                                        \
  case n:                                                                           \
    rows::launch_tail_rows<float, n>(*reinterpret_cast<const TailView<float> *>(&v), st); \
    return;
      BM_ROWS_NB_LIST(X)
#undef X
      case 48:
        rows::launch_tail_rows_w<float, 48>(*reinterpret_cast<const TailView<float> *>(&v), st);
        return;
    }
  }
  switch (v.nb) {
#define X(n)                           \
  case n:                              \
    tail::launch_tail_nb<T, n>(v, st, sc, ev); \
    break;
    BM_TAIL_NB_LIST(X)
#undef X
  }
}
template void tail_factor_launch<double>(const TailView<double> &, cudaStream_t, const TailSched *, cudaEvent_t *);
template void tail_factor_launch<float>(const TailView<float> &, cudaStream_t, const TailSched *, cudaEvent_t *);

// FP64 tails: grid-wide levels [lo, hi) of the tails in v, then the top
// kernel if top (a part of the factor, for pipelined callers).
void tail_factor_launch_range(const TailView<double> &v, cudaStream_t st, const TailSched *sc, int lo, int hi,
                              bool top) {
  switch (v.nb) {
#define X(n)                                                        \
  case n:                                                           \
    tail::launch_tail_range<double, n>(v, st, sc, lo, hi, top, nullptr); \
    break;
    BM_TAIL_NB_LIST(X)
#undef X
  }
}

void tail_default_schedule(int S, int N, int nb, TailSched *sc) {
  sc->top = top_level(N);
  for (int l = 0; l < 32; ++l) {
    if (l < sc->top) {
      const int E = level_elims(N, l);
      const int G = l == 0 ? 0 : ((N - 1) >> (l + 1)) + 1;
      sc->team[l] = tail::pick_team((long)S * (E + G), nb);
    } else {
      sc->team[l] = 0;
    }
  }
}

// Autotuner of the FP64 tail factor's launch schedule, on the caller's
// inputs. The arithmetic of every block element is done by one thread in a
// fixed order whatever the team size or the top level, so every candidate
// gives the same bits and only the time differs.
//  1. Each compiled team size in turn for every grid-wide level (default
//     top level), two runs, per-level event times; each level keeps its
//     fastest team.
//  2. The top level moved one level down or up from the default (one level
//     more or fewer in the per-tail kernel), whole-factor times, two runs.
bool tail_factor_tune(const TailView<double> &v, cudaStream_t st, TailSched *best) {
  if (!tail_nb_supported(v.nb)) return false;
  const int N = v.N, nb = v.nb;
  tail_default_schedule(v.S, N, nb, best);
  const int T0 = best->top;
  cudaEvent_t ev[34];
  for (int k = 0; k < 34; ++k)
    if (cudaEventCreate(&ev[k]) != cudaSuccess) {
      for (int j = 0; j < k; ++j) cudaEventDestroy(ev[j]);
      cudaGetLastError();
      return false;
    }
  const int tmin = nb <= 16 ? 8 : nb <= 32 ? 16 : 32, tmax = nb <= 4 ? 32 : nb <= 16 ? 64 : 128;
  float best_ms[32];
  for (int l = 0; l < 32; ++l) best_ms[l] = 1e30f;
  bool ok = true;
  for (int t = tmin; t <= tmax && ok; t *= 2) {
    TailSched sc = *best;
    for (int l = 0; l < T0; ++l) sc.team[l] = t;
    for (int rep = 0; rep < 2 && ok; ++rep) {
      tail_factor_launch<double>(v, st, &sc, ev);
      ok = cudaStreamSynchronize(st) == cudaSuccess;
      for (int l = 0; l < T0 && ok; ++l) {
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, ev[l], ev[l + 1]);
        if (ms < best_ms[l]) {
          best_ms[l] = ms;
          best->team[l] = t;
        }
      }
    }
  }
  // where the per-tail kernel takes over
  TailSched cand[3];
  int nc = 0;
  for (int d = -1; d <= 1 && ok; ++d) {
    const int top = T0 + d;
    if (top < 0 || top > v.Lc) continue;
    TailSched sc;
    tail_default_schedule(v.S, N, nb, &sc);
    sc.top = top;
    for (int l = 0; l < top; ++l) sc.team[l] = l < T0 ? best->team[l] : sc.team[l];
    if (top > T0) {   // the extra grid-wide level keeps the rule's team
      const int E = level_elims(N, T0), G = T0 == 0 ? 0 : ((N - 1) >> (T0 + 1)) + 1;
      sc.team[T0] = tail::pick_team((long)v.S * (E + G), nb);
    }
    for (int l = top; l < 32; ++l) sc.team[l] = 0;
    cand[nc++] = sc;
  }
  float cbest = 1e30f;
  int ci = -1;
  for (int c = 0; c < nc && ok; ++c) {
    for (int rep = 0; rep < 2 && ok; ++rep) {
      tail_factor_launch<double>(v, st, &cand[c], ev);
      ok = cudaStreamSynchronize(st) == cudaSuccess;
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, ev[0], ev[cand[c].top + 1]);
      if (ok && ms < cbest) {
        cbest = ms;
        ci = c;
      }
    }
  }
  for (int k = 0; k < 34; ++k) cudaEventDestroy(ev[k]);
  if (!ok || ci < 0) {
    cudaGetLastError();
    tail_default_schedule(v.S, N, nb, best);
    return false;
  }
  *best = cand[ci];
  return true;
}

}  // namespace bm
