// C ABI of the library (include/bm.h): the one-time analysis that plans and
// allocates (Sec. V), factor/solve entry points that replay CUDA graphs
// captured per set of pointers (Sec. V: factor and solve pipelines are
// captured separately), status handling and the host-buffer convenience
// entry.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "bm_internal.cuh"

namespace bm {
size_t f64_factor_smem(int nb, int nr);
cudaError_t f64_prepare(int nb, int nr);
void f64_launch_factor(const F64View &v, cudaStream_t st, const TailSched *sc = nullptr);
bool f64_tune(const F64View &v, cudaStream_t st, TailSched *out);
bool tune_cache_lookup(const std::string &key, std::vector<int> &vals);
void tune_cache_store(const std::string &key, const std::vector<int> &vals);
void f64_launch_solve(const F64View &v, const double *r, double *x, double *r0t, cudaStream_t st);
void f64_launch_export_ld(const F64View &v, double *Ld, cudaStream_t st);
void f64_launch_factor_part(const F64View &v, int s0, int s1, int lo, int hi, bool top, cudaStream_t st,
                            const TailSched *sc);

// mixed precision path (bm_mixed.cu)
struct MixedState;
size_t mixed_bytes(int S, int N, int nb, int nr, int cmode, int ff);
bool mixed_ff_residual(double tol, unsigned flags);
bool mixed_ffres(const MixedState *m);
void mixed_launch_residual(MixedState *m, const double *r, const double *x, double *rho, cudaStream_t st);
cudaError_t mixed_prepare(int nb, int nr);
MixedState *mixed_create(int S, int N, int nb, int nr, int cmode, int ff, void *base, size_t bytes, Status *status,
                         unsigned *tickets, cudaStream_t init_stream, bool sync_init);
void mixed_destroy(MixedState *m);
void mixed_launch_factor(MixedState *m, const double *D, const double *E, const double *C, const double *R,
                         cudaStream_t st);
// body_st non-null: st is capturing, and the refinement loop becomes a
// conditional graph node whose body is captured from body_st (programmatic
// launches inside the body when body_pdl is set).
cudaError_t mixed_launch_solve(MixedState *m, const double *r, double *x, int max_refine, double tol,
                               cudaStream_t st, cudaStream_t body_st, cudaStream_t if_st, cudaStream_t body2_st,
                               bool body_pdl);
void mixed_launch_export(MixedState *m, double *Ld, double *Ll, double *Lr, double *F, double *LR,
                         cudaStream_t st);
}  // namespace bm

using namespace bm;

// Chunks of tails whose host-to-device copies the pipelined host entry
// overlaps with the factor (measured on GB300, mixed workload, copies
// 2.93 ms: 2 chunks 8.76 ms per call, 4: 8.22, 8: 7.93, 16: 9.26; serial
// 10.0 ms).
static constexpr int kHostChunks = 8;

struct GraphSlot {
  cudaGraphExec_t exec = nullptr;
  const void *key[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
};

struct bm_handle_s {
  bm_desc desc;
  int Lc = 0;
  int device = 0;
  void *pool = nullptr;
  size_t pool_bytes = 0;
  bool owns_pool = true;
  F64View v{};           // FP64 buffers (unused pointers null in mixed mode)
  double *r0t = nullptr; // [nr] root right-hand side scratch
  Status *status = nullptr;
  unsigned *tickets = nullptr;
  MixedState *mixed = nullptr;
  cudaStream_t cap = nullptr;      // private capture stream
  cudaStream_t cap_body = nullptr; // captures the body of the refinement loop (mixed path)
  cudaStream_t cap_if = nullptr;   // automatic mode: the conditional resumed refinement
  cudaStream_t cap_body2 = nullptr; // and its loop body
  bool loop_pdl = true;            // programmatic launches inside that body (cleared if they do not instantiate)
  GraphSlot gfac, gsol;
  bool factored = false;
  // FP64 tail factor's launch schedule: -1 = the default rule (not tuned),
  // 0 = tuned on this handle's first factor, 1 = taken from the tune cache
  TailSched sched{};
  int sched_src = -1;
  bool sched_ready = false;
  // host-entry staging (allocated on first use)
  double *sD = nullptr, *sE = nullptr, *sC = nullptr, *sR = nullptr, *sr = nullptr, *sx = nullptr;
  // pipelined host entry (FP64): copy stream, its events (fork, one per
  // chunk of tails, the rest of the inputs) and the captured factor
  cudaStream_t cp_st = nullptr;
  cudaEvent_t ev_cp[kHostChunks + 2] = {};
  bool pipe_failed = false;
  bool pipe_last = false;   // the last host-entry call was pipelined
  GraphSlot ghost;
};

static bool valid_desc(const bm_desc *d) {
  if (!d) return false;
  if (d->S < 1 || d->N < 1 || d->nb < 1 || d->nr < 1) return false;
  if (d->nb > 64 || d->nr > 64 || d->S > 65535) return false;
  if (d->N > (1 << 24)) return false;
  if (d->precision != BM_PREC_FP64 && d->precision != BM_PREC_FP32_IR) return false;
  if ((d->flags & BM_FLAG_COUPLING_REFINE) && (d->flags & BM_FLAG_COUPLING_FP32)) return false;
  return true;
}

// Coupling-column mode of the mixed path: 0 = FP32-based root, 1 = automatic,
// 2 = always refine.
static int coupling_mode(const bm_desc *d) {
  if (d->flags & BM_FLAG_COUPLING_FP32) return 0;
  if (d->flags & BM_FLAG_COUPLING_REFINE) return 2;
  return 1;
}

// Float-float refinement residual of the mixed path (1) or FP64 (0): by the
// tolerance (<= 0 means the default 1e-10) and BM_FLAG_RESIDUAL_FP64.
static int ff_mode(const bm_desc *d) {
  return mixed_ff_residual(d->tol > 0.0 ? d->tol : 1e-10, d->flags) ? 1 : 0;
}

static size_t f64_bytes(int S, int N, int nb, int nr) {
  const size_t SN = (size_t)S * N, b2 = (size_t)nb * nb;
  size_t t = 0;
  t += align_up(SN * b2 * sizeof(double), 256) * 5;          // Ld Ll Lr Dt W
  t += align_up((size_t)S * nr * nb * sizeof(double), 256);  // F
  t += align_up((size_t)S * nr * nr * sizeof(double), 256);  // U
  t += align_up((size_t)nr * nr * sizeof(double), 256) * 2;  // LR Rt
  t += align_up(SN * nb * sizeof(double), 256) * 3;          // invd y zt
  t += align_up((size_t)S * nr * sizeof(double), 256);       // tb
  t += align_up((size_t)nr * sizeof(double), 256);           // r0t
  return t;
}

static const size_t kHeader = 512;   // status + tickets

extern "C" int bm_version(void) { return BM_VERSION; }

extern "C" const char *bm_status_string(bm_status s) {
  switch (s) {
    case BM_OK: return "ok";
    case BM_ERR_INVALID_ARG: return "invalid argument";
    case BM_ERR_NOT_SPD: return "matrix is not symmetric positive definite (non-positive pivot)";
    case BM_ERR_OOM: return "device allocation failed";
    case BM_ERR_CUDA: return "CUDA runtime error";
    case BM_ERR_NOT_CONVERGED: return "iterative refinement did not reach the tolerance";
    case BM_ERR_TIMEOUT: return "bounded device wait timed out";
    case BM_ERR_NOT_FACTORED: return "solve called before factor";
  }
  return "unknown status";
}

extern "C" size_t bm_workspace_bytes(const bm_desc *d) {
  if (!valid_desc(d)) return 0;
  size_t t = kHeader;
  if (d->precision == BM_PREC_FP64)
    t += f64_bytes(d->S, d->N, d->nb, d->nr);
  else
    t += mixed_bytes(d->S, d->N, d->nb, d->nr, coupling_mode(d), ff_mode(d));
  return t;
}

// Builds a handle over `mem` (bytes >= bm_workspace_bytes) or, when mem is
// null, over memory it allocates and owns. light = true skips the graph
// capture stream and every synchronizing call (used by the serving loop,
// which launches without graphs on its own streams); initialization is then
// ordered on init_stream.
bm_status analyze_impl(const bm_desc *desc, void *mem, size_t bytes, cudaStream_t init_stream, bool light,
                       bm_handle *out) {
  if (!out) return BM_ERR_INVALID_ARG;
  *out = nullptr;
  if (!valid_desc(desc)) return BM_ERR_INVALID_ARG;
  const size_t need = bm_workspace_bytes(desc);
  if (mem && bytes < need) return BM_ERR_INVALID_ARG;
  bm_handle h = new (std::nothrow) bm_handle_s();
  if (!h) return BM_ERR_OOM;
  h->desc = *desc;
  if (h->desc.max_refine <= 0) h->desc.max_refine = 10;
  if (!(h->desc.tol > 0.0)) h->desc.tol = 1e-10;
  if (light) h->desc.flags |= BM_FLAG_NO_GRAPH;
  const int S = desc->S, N = desc->N, nb = desc->nb, nr = desc->nr;
  h->Lc = chain_levels(N);
  cudaGetDevice(&h->device);
  h->pool_bytes = need;
  if (mem) {
    h->pool = mem;
    h->owns_pool = false;
  } else if (cudaMalloc(&h->pool, h->pool_bytes) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return BM_ERR_OOM;
  }
  if (light ? cudaMemsetAsync(h->pool, 0, kHeader, init_stream) != cudaSuccess
            : cudaMemset(h->pool, 0, kHeader) != cudaSuccess)
    goto cuda_fail;
  h->status = (Status *)h->pool;
  h->tickets = (unsigned *)((char *)h->pool + 256);
  if (desc->precision == BM_PREC_FP64) {
    char *p = (char *)h->pool + kHeader;
    const size_t SN = (size_t)S * N, b2 = (size_t)nb * nb;
    auto take = [&](size_t nbytes) {
      double *q = (double *)p;
      p += align_up(nbytes, 256);
      return q;
    };
    F64View &v = h->v;
    v.S = S; v.N = N; v.nb = nb; v.nr = nr; v.Lc = h->Lc;
    v.Ld = take(SN * b2 * 8); v.Ll = take(SN * b2 * 8); v.Lr = take(SN * b2 * 8);
    v.Dt = take(SN * b2 * 8); v.W = take(SN * b2 * 8);
    v.F = take((size_t)S * nr * nb * 8); v.U = take((size_t)S * nr * nr * 8);
    v.LR = take((size_t)nr * nr * 8); v.Rt = take((size_t)nr * nr * 8);
    v.invd = take(SN * nb * 8); v.y = take(SN * nb * 8); v.zt = take(SN * nb * 8);
    v.tb = take((size_t)S * nr * 8);
    h->r0t = take((size_t)nr * 8);
    v.tickets = h->tickets;
    v.status = h->status;
    if (f64_prepare(nb, nr) != cudaSuccess) goto cuda_fail;
  } else {
    if (mixed_prepare(nb, nr) != cudaSuccess) goto cuda_fail;
    h->mixed = mixed_create(S, N, nb, nr, coupling_mode(desc), ff_mode(desc), (char *)h->pool + kHeader, h->pool_bytes - kHeader, h->status,
                            h->tickets, light ? init_stream : nullptr, !light);
    if (!h->mixed) goto cuda_fail;
  }
  if (!light) {
    if (cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess) goto cuda_fail;
    if (h->mixed && (cudaStreamCreateWithFlags(&h->cap_body, cudaStreamNonBlocking) != cudaSuccess ||
                     cudaStreamCreateWithFlags(&h->cap_if, cudaStreamNonBlocking) != cudaSuccess ||
                     cudaStreamCreateWithFlags(&h->cap_body2, cudaStreamNonBlocking) != cudaSuccess))
      goto cuda_fail;
    if (cudaDeviceSynchronize() != cudaSuccess) goto cuda_fail;
  }
  *out = h;
  return BM_OK;
cuda_fail:
  cudaGetLastError();
  if (h->mixed) mixed_destroy(h->mixed);
  if (h->cap) cudaStreamDestroy(h->cap);
  if (h->cap_body) cudaStreamDestroy(h->cap_body);
  if (h->cap_if) cudaStreamDestroy(h->cap_if);
  if (h->cap_body2) cudaStreamDestroy(h->cap_body2);
  if (h->owns_pool) cudaFree(h->pool);
  delete h;
  return BM_ERR_CUDA;
}

extern "C" bm_status bm_analyze(const bm_desc *desc, void *stream, bm_handle *out) {
  (void)stream;
  return analyze_impl(desc, nullptr, 0, nullptr, false, out);
}

// Releases a handle built by analyze_impl without synchronizing the device
// (the caller guarantees its work has finished).
void release_impl(bm_handle h) {
  if (!h) return;
  if (h->gfac.exec) cudaGraphExecDestroy(h->gfac.exec);
  if (h->gsol.exec) cudaGraphExecDestroy(h->gsol.exec);
  if (h->ghost.exec) cudaGraphExecDestroy(h->ghost.exec);
  for (cudaEvent_t ev : h->ev_cp)
    if (ev) cudaEventDestroy(ev);
  if (h->cp_st) cudaStreamDestroy(h->cp_st);
  if (h->mixed) mixed_destroy(h->mixed);
  if (h->cap) cudaStreamDestroy(h->cap);
  if (h->cap_body) cudaStreamDestroy(h->cap_body);
  if (h->cap_if) cudaStreamDestroy(h->cap_if);
  if (h->cap_body2) cudaStreamDestroy(h->cap_body2);
  if (h->sD) cudaFree(h->sD);
  if (h->owns_pool) cudaFree(h->pool);
  delete h;
}

Status *handle_status(bm_handle h) { return h->status; }

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

static bool key_match(const GraphSlot &g, const void *const *k, int n) {
  if (!g.exec) return false;
  for (int i = 0; i < n; ++i)
    if (g.key[i] != k[i]) return false;
  return true;
}

// body(stream, capturing) issues the work; it returns void (errors are read
// from the runtime's last error) or a cudaError_t.
template <typename Body>
static cudaError_t call_body(Body &body, cudaStream_t s, bool capturing) {
  if constexpr (std::is_void_v<decltype(body(s, capturing))>) {
    body(s, capturing);
    return cudaPeekAtLastError();
  } else {
    return body(s, capturing);
  }
}

// Runs body either directly or through the graph cached in slot
// (re-captured on the handle's private stream when the pointers change).
// A capture during which any call failed is discarded.
template <typename Body>
static bm_status run(bm_handle h, GraphSlot &slot, const void *const *key, int nkey, cudaStream_t st,
                     Body body) {
  if (h->desc.flags & BM_FLAG_NO_GRAPH) {
    const cudaError_t e = call_body(body, st, false);
    cudaGetLastError();
    return e == cudaSuccess ? BM_OK : BM_ERR_CUDA;
  }
  if (!key_match(slot, key, nkey)) {
    if (slot.exec) {
      cudaGraphExecDestroy(slot.exec);
      slot.exec = nullptr;
    }
    cudaGetLastError();
    if (cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return BM_ERR_CUDA;
    const cudaError_t eb = call_body(body, h->cap, true);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->cap, &g);
    if (eb != cudaSuccess || e != cudaSuccess || !g) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return BM_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&slot.exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      cudaGetLastError();
      slot.exec = nullptr;
      return BM_ERR_CUDA;
    }
    for (int i = 0; i < nkey; ++i) slot.key[i] = key[i];
  }
  return cudaGraphLaunch(slot.exec, st) == cudaSuccess ? BM_OK : BM_ERR_CUDA;
}

// The FP64 factor's launch schedule, once per handle: from the tune cache
// (keyed by GPU and system shape), else tuned on these inputs (the stream
// is synchronized; the tuning runs are full factors, overwritten by the
// factor that follows), unless BM_FLAG_NO_TUNE or BM_FLAG_NO_GRAPH asks for
// the default rule.
static void prepare_schedule(bm_handle h, const F64View &v, cudaStream_t st) {
  const bm_desc &d = h->desc;
  tail_default_schedule(d.S, d.N, d.nb, &h->sched);
  h->sched_src = -1;
  h->sched_ready = true;
  if ((d.flags & (BM_FLAG_NO_TUNE | BM_FLAG_NO_GRAPH)) || !tail_nb_supported(d.nb)) return;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, h->device) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  char kb[320];
  snprintf(kb, sizeof kb, "fp64-schedule|%.200s|S=%d|N=%d|nb=%d|nr=%d", prop.name, d.S, d.N, d.nb, d.nr);
  std::vector<int> vals;
  if (tune_cache_lookup(kb, vals) && (int)vals.size() == 1 + (vals.empty() ? 0 : vals[0]) && vals[0] >= 0 &&
      vals[0] <= h->Lc && vals[0] < 32) {
    h->sched.top = vals[0];
    for (int l = 0; l < 32; ++l) h->sched.team[l] = l < vals[0] ? vals[1 + l] : 0;
    h->sched_src = 1;
    return;
  }
  TailSched t;
  if (!f64_tune(v, st, &t)) return;
  h->sched = t;
  h->sched_src = 0;
  vals.assign(1, t.top);
  for (int l = 0; l < t.top; ++l) vals.push_back(t.team[l]);
  tune_cache_store(kb, vals);
}

extern "C" bm_status bm_factor(bm_handle h, const double *D, const double *E, const double *C,
                               const double *R, void *stream) {
  if (!h || !D || !C || !R || (h->desc.N > 1 && !E)) return BM_ERR_INVALID_ARG;
  if (!aligned16(D) || !aligned16(C) || !aligned16(R) || (E && !aligned16(E))) return BM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const void *key[4] = {D, E, C, R};
  bm_status s;
  if (h->mixed) {
    MixedState *m = h->mixed;
    Status *status = h->status;
    s = run(h, h->gfac, key, 4, st, [&](cudaStream_t cs, bool) {
      cudaMemsetAsync(status, 0, sizeof(Status), cs);
      mixed_launch_factor(m, D, E, C, R, cs);
    });
  } else {
    F64View v = h->v;
    v.D = D; v.E = E; v.C = C; v.R = R;
    if (!h->sched_ready) prepare_schedule(h, v, st);
    const TailSched *sc = &h->sched;
    s = run(h, h->gfac, key, 4, st, [&](cudaStream_t cs, bool) {
      cudaMemsetAsync(v.status, 0, sizeof(Status), cs);
      f64_launch_factor(v, cs, sc);
    });
    h->v.D = D; h->v.E = E; h->v.C = C; h->v.R = R;
  }
  if (s == BM_OK) h->factored = true;
  return s;
}

extern "C" bm_status bm_solve(bm_handle h, const double *r, double *x, void *stream) {
  if (!h || !r || !x || (const void *)r == (const void *)x) return BM_ERR_INVALID_ARG;
  if (!aligned16(r) || !aligned16(x)) return BM_ERR_INVALID_ARG;
  if (!h->factored) return BM_ERR_NOT_FACTORED;
  cudaStream_t st = (cudaStream_t)stream;
  if (h->mixed) {
    MixedState *m = h->mixed;
    const int mr = h->desc.max_refine;
    const double tol = h->desc.tol;
    // the refinement residual reads the factor's inputs: key on them as well
    const void *key[6] = {r, x, h->gfac.key[0], h->gfac.key[1], h->gfac.key[2], h->gfac.key[3]};
    cudaStream_t body_st = h->cap_body;
    auto body = [&](cudaStream_t cs, bool capturing) {
      return mixed_launch_solve(m, r, x, mr, tol, cs, capturing ? body_st : nullptr, capturing ? h->cap_if : nullptr,
                                capturing ? h->cap_body2 : nullptr, h->loop_pdl);
    };
    bm_status s = run(h, h->gsol, key, 6, st, body);
    if (s == BM_ERR_CUDA && h->loop_pdl && !(h->desc.flags & BM_FLAG_NO_GRAPH)) {
      // a graph whose loop body chains its kernels programmatically may not
      // instantiate on every driver: capture the body with plain launches
      h->loop_pdl = false;
      s = run(h, h->gsol, key, 6, st, body);
    }
    return s;
  }
  F64View v = h->v;
  double *r0t = h->r0t;
  const void *key[2] = {r, x};
  return run(h, h->gsol, key, 2, st, [&](cudaStream_t cs, bool) { f64_launch_solve(v, r, x, r0t, cs); });
}

extern "C" bm_status bm_residual(bm_handle h, const double *r, const double *x, double *rho, void *stream) {
  if (!h || !r || !x || !rho || !h->mixed) return BM_ERR_INVALID_ARG;
  if (!aligned16(r) || !aligned16(x) || !aligned16(rho)) return BM_ERR_INVALID_ARG;
  if ((const void *)rho == (const void *)r || (const void *)rho == (const void *)x) return BM_ERR_INVALID_ARG;
  if (!h->factored) return BM_ERR_NOT_FACTORED;
  mixed_launch_residual(h->mixed, r, x, rho, (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? BM_OK : BM_ERR_CUDA;
}

extern "C" bm_status bm_schedule(bm_handle h, int *top_level, int *team_per_level, int *source) {
  if (!h) return BM_ERR_INVALID_ARG;
  if (h->mixed || !tail_nb_supported(h->desc.nb)) return BM_ERR_INVALID_ARG;
  if (!h->sched_ready) return BM_ERR_NOT_FACTORED;
  if (top_level) *top_level = h->sched.top;
  if (team_per_level)
    for (int l = 0; l < 32; ++l) team_per_level[l] = l < h->sched.top ? h->sched.team[l] : 0;
  if (source) *source = h->sched_src;
  return BM_OK;
}

extern "C" bm_status bm_query(bm_handle h, void *stream, bm_info *info) {
  if (!h) return BM_ERR_INVALID_ARG;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
    cudaGetLastError();
    return BM_ERR_CUDA;
  }
  Status st;
  if (cudaMemcpy(&st, h->status, sizeof(Status), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return BM_ERR_CUDA;
  }
  if (info) {
    info->status = st.code;
    info->fail_scenario = st.code == BM_ERR_NOT_SPD ? st.scenario : 0;
    info->fail_stage = st.code == BM_ERR_NOT_SPD ? st.stage : 0;
    info->iters = h->mixed ? st.iters : 0;
    info->backward_error = h->mixed ? st.eta : -1.0;
    info->coupling_refined = h->mixed ? st.coupled : 0;
    info->residual_float_float = h->mixed && mixed_ffres(h->mixed) && !st.ffbad ? 1 : 0;
    info->host_pipelined = h->pipe_last ? 1 : 0;
  }
  return (bm_status)st.code;
}

extern "C" bm_status bm_export_factor(bm_handle h, double *Ld, double *Ll, double *Lr, double *F,
                                      double *LR, void *stream) {
  if (!h) return BM_ERR_INVALID_ARG;
  if (!h->factored) return BM_ERR_NOT_FACTORED;
  cudaStream_t st = (cudaStream_t)stream;
  if (h->mixed) {
    mixed_launch_export(h->mixed, Ld, Ll, Lr, F, LR, st);
    return cudaGetLastError() == cudaSuccess ? BM_OK : BM_ERR_CUDA;
  }
  const F64View &v = h->v;
  const size_t bb = (size_t)v.S * v.N * v.nb * v.nb * sizeof(double);
  cudaError_t e = cudaSuccess;
  if (Ld && e == cudaSuccess) {
    f64_launch_export_ld(v, Ld, st);
    e = cudaGetLastError();
  }
  if (Ll && e == cudaSuccess) e = cudaMemcpyAsync(Ll, v.Ll, bb, cudaMemcpyDeviceToDevice, st);
  if (Lr && e == cudaSuccess) e = cudaMemcpyAsync(Lr, v.Lr, bb, cudaMemcpyDeviceToDevice, st);
  if (F && e == cudaSuccess)
    e = cudaMemcpyAsync(F, v.F, (size_t)v.S * v.nr * v.nb * sizeof(double), cudaMemcpyDeviceToDevice, st);
  if (LR && e == cudaSuccess)
    e = cudaMemcpyAsync(LR, v.LR, (size_t)v.nr * v.nr * sizeof(double), cudaMemcpyDeviceToDevice, st);
  return e == cudaSuccess ? BM_OK : BM_ERR_CUDA;
}

static bool host_pinned(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

// The factor of the host entry with its copies pipelined (FP64 tails with
// compile-time kernels, a schedule already chosen, page-locked inputs): the
// tails' blocks are copied in kHostChunks chunks on a second stream, and the
// first grid-wide level of a chunk runs as soon as its blocks have arrived,
// so the transfer of later chunks overlaps the factor of earlier ones (one
// chunk's level 0 takes about as long as its copy; running level 1 per
// chunk as well measured slower: 8.97 against 7.93 ms per call on the mixed
// workload, the smaller level-1 grids filling the SMs less well). The
// remaining levels run over all tails once the last chunk has arrived, and
// the top kernel (whose last CTA does the root step) once C, R and r have. Every block
// is computed by the same kernels in the same order as in bm_factor, so the
// factor is bitwise that of the device entry. Returns false when the
// pipelined form does not apply or could not be issued; the caller then
// copies and factors serially.
static bool factor_host_pipelined(bm_handle h, const double *hD, const double *hE, const double *hC,
                                  const double *hR, const double *hr, cudaStream_t st, bm_status *out) {
  const bm_desc &d = h->desc;
  if (h->mixed || h->pipe_failed || !h->sched_ready || !tail_nb_supported(d.nb) || d.S < 2) return false;
  if (!h->cap && !(d.flags & BM_FLAG_NO_GRAPH)) return false;
  if (!host_pinned(hD) || !host_pinned(hC) || !host_pinned(hR) || !host_pinned(hr) ||
      (d.N > 1 && !host_pinned(hE)))
    return false;
  if (!h->cp_st) {
    bool ok = cudaStreamCreateWithFlags(&h->cp_st, cudaStreamNonBlocking) == cudaSuccess;
    for (int i = 0; ok && i < kHostChunks + 2; ++i)
      ok = cudaEventCreateWithFlags(&h->ev_cp[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      h->pipe_failed = true;
      return false;
    }
  }
  const int S = d.S, N = d.N, nb = d.nb, nr = d.nr;
  const size_t b2 = (size_t)nb * nb, n = (size_t)S * N * nb + nr;
  const int K = S < kHostChunks ? S : kHostChunks;
  const int lp = h->sched.top < 1 ? h->sched.top : 1;
  F64View v = h->v;
  v.D = h->sD; v.E = N > 1 ? h->sE : nullptr; v.C = h->sC; v.R = h->sR;
  const TailSched *sc = &h->sched;
  const cudaMemcpyKind H2D = cudaMemcpyHostToDevice;
  const void *key[5] = {hD, hE, hC, hR, hr};
  *out = run(h, h->ghost, key, 5, st, [&](cudaStream_t cs, bool) -> cudaError_t {
    cudaStream_t cp = h->cp_st;
    cudaError_t e = cudaMemsetAsync(v.status, 0, sizeof(Status), cs);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_cp[0], cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cp, h->ev_cp[0], 0);
    for (int c = 0; c < K && e == cudaSuccess; ++c) {
      const size_t s0 = (size_t)S * c / K, s1 = (size_t)S * (c + 1) / K;
      e = cudaMemcpyAsync(h->sD + s0 * N * b2, hD + s0 * N * b2, (s1 - s0) * N * b2 * 8, H2D, cp);
      if (e == cudaSuccess && N > 1)
        e = cudaMemcpyAsync(h->sE + s0 * (N - 1) * b2, hE + s0 * (N - 1) * b2, (s1 - s0) * (N - 1) * b2 * 8, H2D,
                            cp);
      if (e == cudaSuccess) e = cudaEventRecord(h->ev_cp[1 + c], cp);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->sC, hC, (size_t)S * nr * nb * 8, H2D, cp);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->sR, hR, (size_t)nr * nr * 8, H2D, cp);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->sr, hr, n * 8, H2D, cp);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_cp[K + 1], cp);
    for (int c = 0; c < K && e == cudaSuccess; ++c) {
      e = cudaStreamWaitEvent(cs, h->ev_cp[1 + c], 0);
      if (e == cudaSuccess && lp > 0)
        f64_launch_factor_part(v, (int)((long)S * c / K), (int)((long)S * (c + 1) / K), 0, lp, false, cs, sc);
    }
    // the later levels need only the blocks; C, R and r (copied last) are
    // first read by the top kernel
    if (e == cudaSuccess) f64_launch_factor_part(v, 0, S, lp, 1 << 30, false, cs, sc);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, h->ev_cp[K + 1], 0);
    if (e == cudaSuccess) f64_launch_factor_part(v, 0, S, 1 << 30, 1 << 30, true, cs, sc);
    return e == cudaSuccess ? cudaPeekAtLastError() : e;
  });
  if (*out != BM_OK) {
    // a form that cannot be captured or launched here is not tried again:
    // once the copy stream is idle, this call and later ones take the
    // serial form
    h->pipe_failed = true;
    cudaStreamSynchronize(h->cp_st);
    cudaGetLastError();
    return false;
  }
  h->v.D = v.D; h->v.E = v.E; h->v.C = v.C; h->v.R = v.R;
  h->factored = true;
  return true;
}

extern "C" bm_status bm_factor_solve_host(bm_handle h, const double *hD, const double *hE, const double *hC,
                                          const double *hR, const double *hr, double *hx, void *stream) {
  if (!h || !hD || !hC || !hR || !hr || !hx || (h->desc.N > 1 && !hE)) return BM_ERR_INVALID_ARG;
  const int S = h->desc.S, N = h->desc.N, nb = h->desc.nb, nr = h->desc.nr;
  const size_t nD = (size_t)S * N * nb * nb, nE = (size_t)S * (N - 1) * nb * nb;
  const size_t nC = (size_t)S * nr * nb, nR = (size_t)nr * nr, n = (size_t)S * N * nb + nr;
  if (!h->sD) {
    void *p = nullptr;
    const size_t bytes = align_up(nD * 8, 256) + align_up((nE ? nE : 1) * 8, 256) + align_up(nC * 8, 256) +
                         align_up(nR * 8, 256) + 2 * align_up(n * 8, 256);
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return BM_ERR_OOM;
    }
    char *c = (char *)p;
    h->sD = (double *)c; c += align_up(nD * 8, 256);
    h->sE = (double *)c; c += align_up((nE ? nE : 1) * 8, 256);
    h->sC = (double *)c; c += align_up(nC * 8, 256);
    h->sR = (double *)c; c += align_up(nR * 8, 256);
    h->sr = (double *)c; c += align_up(n * 8, 256);
    h->sx = (double *)c;
  }
  cudaStream_t st = (cudaStream_t)stream;
  bm_status s = BM_OK;
  h->pipe_last = factor_host_pipelined(h, hD, hE, hC, hR, hr, st, &s);
  if (!h->pipe_last) {
    cudaError_t e = cudaMemcpyAsync(h->sD, hD, nD * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && nE) e = cudaMemcpyAsync(h->sE, hE, nE * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->sC, hC, nC * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->sR, hR, nR * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->sr, hr, n * 8, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return BM_ERR_CUDA;
    }
    s = bm_factor(h, h->sD, nE ? h->sE : nullptr, h->sC, h->sR, stream);
  }
  if (s != BM_OK) return s;
  s = bm_solve(h, h->sr, h->sx, stream);
  if (s != BM_OK) return s;
  if (cudaMemcpyAsync(hx, h->sx, n * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess) {
    cudaGetLastError();
    return BM_ERR_CUDA;
  }
  return bm_query(h, stream, nullptr);
}

extern "C" void bm_destroy(bm_handle h) {
  if (!h) return;
  cudaDeviceSynchronize();
  release_impl(h);
  cudaGetLastError();
}
