// Serving runtime (include/bm.h, "Serving runtime"): a first-in first-out
// request loop over a device arena and a fixed set of stream slots. Every
// admitted request gets a handle built over its arena range (no allocation,
// no graph, no device synchronization), is factored once (Alg. 1) and solved
// for each of its right-hand sides (Alg. 2) on its slot's stream, so that
// requests admitted at different times overlap on the GPU. Completion is
// detected with events; the status words are copied to page-locked host
// memory in stream order, so retiring a request never synchronizes.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <chrono>
#include <deque>
#include <iterator>
#include <map>
#include <new>
#include <vector>

#include "bm_internal.cuh"

using namespace bm;

bm_status analyze_impl(const bm_desc *desc, void *mem, size_t bytes, cudaStream_t init_stream, bool light,
                       bm_handle *out);
void release_impl(bm_handle h);
Status *handle_status(bm_handle h);

namespace {

constexpr size_t kAlign = 256;

// First-fit allocator over [0, cap) with coalescing of free neighbours.
class Arena {
 public:
  explicit Arena(size_t cap) : cap_(cap) { free_[0] = cap; }
  // Returns the offset of a range of `bytes` (a multiple of kAlign), or
  // SIZE_MAX when no free range is large enough.
  size_t alloc(size_t bytes) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      const size_t off = it->first, rest = it->second - bytes;
      free_.erase(it);
      if (rest) free_[off + bytes] = rest;
      used_ += bytes;
      return off;
    }
    return SIZE_MAX;
  }
  void release(size_t off, size_t bytes) {
    used_ -= bytes;
    auto next = free_.lower_bound(off);
    if (next != free_.end() && off + bytes == next->first) {
      bytes += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {
        prev->second += bytes;
        return;
      }
    }
    free_[off] = bytes;
  }
  size_t used() const { return used_; }
  size_t capacity() const { return cap_; }

 private:
  size_t cap_, used_ = 0;
  std::map<size_t, size_t> free_;
};

struct Pending {
  bm_request req;
  double t_submit_us;
  size_t bytes;
  int precision;          // of this attempt
  int fallback;           // 1 for the FP64 re-run of a failed mixed attempt
  double t_first_start_us;
};

// One stream slot. hs[0] receives the status word after the factor, hs[1+j]
// after the j-th solve.
struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t ev_start = nullptr, ev_factor = nullptr, ev_done = nullptr;
  Status *hs = nullptr;
  bool busy = false;
  Pending job{};
  bm_handle h = nullptr;
  size_t off = 0;
};

size_t n_of(const bm_request &q) { return (size_t)q.S * q.N * q.nb + q.nr; }

struct IoLayout {
  size_t work, D, E, C, R, r, x, total;
};

// Offsets (relative to the request's arena range) of the factor workspace
// and, under BM_REQ_HOST_IO, of the staged inputs and outputs.
bool layout_of(const bm_server_desc &sd, int precision, const bm_request &q, IoLayout *L) {
  bm_desc d{};
  d.S = q.S; d.N = q.N; d.nb = q.nb; d.nr = q.nr;
  d.precision = precision;
  d.max_refine = sd.max_refine;
  d.tol = sd.tol;
  const size_t work = bm_workspace_bytes(&d);
  if (!work) return false;
  auto up = [](size_t b) { return (b + kAlign - 1) / kAlign * kAlign; };
  L->work = 0;
  size_t o = up(work);
  if (q.flags & BM_REQ_HOST_IO) {
    const size_t nD = (size_t)q.S * q.N * q.nb * q.nb, nE = (size_t)q.S * (q.N - 1) * q.nb * q.nb;
    const size_t nC = (size_t)q.S * q.nr * q.nb, nR = (size_t)q.nr * q.nr, n = n_of(q) * q.nrhs;
    L->D = o; o += up(nD * 8);
    L->E = o; o += up((nE ? nE : 1) * 8);
    L->C = o; o += up(nC * 8);
    L->R = o; o += up(nR * 8);
    L->r = o; o += up(n * 8);
    L->x = o; o += up(n * 8);
  }
  L->total = o;
  return true;
}

bool valid_request(const bm_server_desc &sd, const bm_request *q) {
  if (!q) return false;
  if (q->nrhs < 1 || q->nrhs > BM_SERVE_MAX_RHS) return false;
  if (q->flags & ~BM_REQ_HOST_IO) return false;
  if (q->S < 1 || q->N < 1 || q->nb < 1 || q->nr < 1) return false;
  if (!q->D || !q->C || !q->R || !q->r || !q->x || (q->N > 1 && !q->E)) return false;
  if (sd.precision == BM_PREC_FP32_IR && !tail_nb_supported(q->nb)) return false;
  const size_t n = n_of(*q) * q->nrhs * sizeof(double);
  const char *r0 = (const char *)q->r, *x0 = (const char *)q->x;
  if (r0 < x0 + n && x0 < r0 + n) return false;   // r and x overlap
  if (!(q->flags & BM_REQ_HOST_IO)) {
    auto al = [](const void *p) { return ((uintptr_t)p & 15u) == 0; };
    if (!al(q->D) || !al(q->C) || !al(q->R) || !al(q->r) || !al(q->x) || (q->E && !al(q->E))) return false;
  }
  return true;
}

double now_us(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

struct bm_server_s {
  bm_server_desc desc{};
  int device = 0;
  char *arena_base = nullptr;
  Arena *arena = nullptr;
  std::vector<Slot> slots;
  Status *host_status = nullptr;
  std::deque<Pending> queue;
  std::deque<bm_completion> done;
  std::chrono::steady_clock::time_point t0;
  cudaEvent_t ev_base = nullptr;
  bm_server_stats stats{};
};

extern "C" size_t bm_server_request_bytes(const bm_server_desc *desc, const bm_request *req) {
  if (!desc || !valid_request(*desc, req)) return 0;
  IoLayout L;
  if (!layout_of(*desc, desc->precision, *req, &L)) return 0;
  return L.total;
}

static bool valid_server_desc(const bm_server_desc *d) {
  if (!d || d->hbm_budget < kAlign) return false;
  if (d->slots < 1 || d->slots > BM_SERVE_MAX_SLOTS) return false;
  if (d->flags & ~BM_SERVE_FP64_FALLBACK) return false;
  return d->precision == BM_PREC_FP64 || d->precision == BM_PREC_FP32_IR;
}

static void free_server(bm_server s) {
  for (Slot &sl : s->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.h) release_impl(sl.h);
    if (sl.ev_start) cudaEventDestroy(sl.ev_start);
    if (sl.ev_factor) cudaEventDestroy(sl.ev_factor);
    if (sl.ev_done) cudaEventDestroy(sl.ev_done);
    if (sl.stream) cudaStreamDestroy(sl.stream);
  }
  if (s->ev_base) cudaEventDestroy(s->ev_base);
  if (s->host_status) cudaFreeHost(s->host_status);
  if (s->arena_base) cudaFree(s->arena_base);
  delete s->arena;
  cudaGetLastError();
  delete s;
}

extern "C" bm_status bm_server_create(const bm_server_desc *desc, bm_server *out) {
  if (!out) return BM_ERR_INVALID_ARG;
  *out = nullptr;
  if (!valid_server_desc(desc)) return BM_ERR_INVALID_ARG;
  bm_server s = new (std::nothrow) bm_server_s();
  if (!s) return BM_ERR_OOM;
  s->desc = *desc;
  if (s->desc.max_refine <= 0) s->desc.max_refine = 10;
  if (!(s->desc.tol > 0.0)) s->desc.tol = 1e-10;
  cudaGetDevice(&s->device);
  const size_t cap = desc->hbm_budget / kAlign * kAlign;
  if (cudaMalloc(&s->arena_base, cap) != cudaSuccess) {
    cudaGetLastError();
    s->arena_base = nullptr;
    free_server(s);
    return BM_ERR_OOM;
  }
  s->arena = new (std::nothrow) Arena(cap);
  s->slots.resize(desc->slots);
  bool ok = s->arena != nullptr;
  ok = ok && cudaHostAlloc((void **)&s->host_status, sizeof(Status) * (BM_SERVE_MAX_RHS + 1) * desc->slots,
                           cudaHostAllocDefault) == cudaSuccess;
  for (int i = 0; ok && i < desc->slots; ++i) {
    Slot &sl = s->slots[i];
    ok = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreate(&sl.ev_start) == cudaSuccess && cudaEventCreate(&sl.ev_factor) == cudaSuccess &&
         cudaEventCreate(&sl.ev_done) == cudaSuccess;
    if (ok) sl.hs = s->host_status + (size_t)i * (BM_SERVE_MAX_RHS + 1);
  }
  // the device clock of every completion is taken relative to ev_base
  ok = ok && cudaEventCreate(&s->ev_base) == cudaSuccess && cudaEventRecord(s->ev_base, s->slots[0].stream) ==
                                                               cudaSuccess &&
       cudaEventSynchronize(s->ev_base) == cudaSuccess;
  s->t0 = std::chrono::steady_clock::now();
  if (!ok) {
    free_server(s);
    return BM_ERR_CUDA;
  }
  s->stats.budget = cap;
  *out = s;
  return BM_OK;
}

// Launches everything of one admitted request on its slot; a status other
// than BM_OK means a launch or copy could not be issued.
static bm_status launch_request(bm_server s, Slot &sl) {
  const bm_request &q = sl.job.req;
  const bm_server_desc &sd = s->desc;
  cudaStream_t st = sl.stream;
  char *base = s->arena_base + sl.off;
  IoLayout L;
  layout_of(sd, sl.job.precision, q, &L);
  bm_desc d{};
  d.S = q.S; d.N = q.N; d.nb = q.nb; d.nr = q.nr;
  d.precision = sl.job.precision;
  d.max_refine = sd.max_refine;
  d.tol = sd.tol;
  d.flags = BM_FLAG_NO_GRAPH;
  if (cudaEventRecord(sl.ev_start, st) != cudaSuccess) return BM_ERR_CUDA;
  bm_status rc = analyze_impl(&d, base + L.work, L.total - L.work, st, true, &sl.h);
  if (rc != BM_OK) return rc;
  const size_t n = n_of(q);
  const double *D = q.D, *E = q.E, *C = q.C, *R = q.R, *r = q.r;
  double *x = q.x;
  if (q.flags & BM_REQ_HOST_IO) {
    const size_t nD = (size_t)q.S * q.N * q.nb * q.nb, nE = (size_t)q.S * (q.N - 1) * q.nb * q.nb;
    const size_t nC = (size_t)q.S * q.nr * q.nb, nR = (size_t)q.nr * q.nr;
    double *dD = (double *)(base + L.D), *dE = (double *)(base + L.E), *dC = (double *)(base + L.C);
    double *dR = (double *)(base + L.R), *dr = (double *)(base + L.r);
    cudaError_t e = cudaMemcpyAsync(dD, q.D, nD * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && nE) e = cudaMemcpyAsync(dE, q.E, nE * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dC, q.C, nC * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dR, q.R, nR * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dr, q.r, n * q.nrhs * 8, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return BM_ERR_CUDA;
    D = dD; E = nE ? dE : nullptr; C = dC; R = dR; r = dr;
    x = (double *)(base + L.x);
  }
  Status *dev_status = handle_status(sl.h);
  rc = bm_factor(sl.h, D, E, C, R, st);
  if (rc != BM_OK) return rc;
  if (cudaMemcpyAsync(&sl.hs[0], dev_status, sizeof(Status), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return BM_ERR_CUDA;
  if (cudaEventRecord(sl.ev_factor, st) != cudaSuccess) return BM_ERR_CUDA;
  for (int j = 0; j < q.nrhs; ++j) {
    rc = bm_solve(sl.h, r + j * n, x + j * n, st);
    if (rc != BM_OK) return rc;
    if (cudaMemcpyAsync(&sl.hs[1 + j], dev_status, sizeof(Status), cudaMemcpyDeviceToHost, st) != cudaSuccess)
      return BM_ERR_CUDA;
  }
  if ((q.flags & BM_REQ_HOST_IO) &&
      cudaMemcpyAsync(q.x, x, n * q.nrhs * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return BM_ERR_CUDA;
  return cudaEventRecord(sl.ev_done, st) == cudaSuccess ? BM_OK : BM_ERR_CUDA;
}

static double event_us(bm_server s, cudaEvent_t e) {
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, s->ev_base, e) != cudaSuccess) {
    cudaGetLastError();
    return -1.0;
  }
  return (double)ms * 1e3;
}

// Builds the completion of a finished (or failed) request and frees its
// slot and arena range.
static void retire(bm_server s, Slot &sl, bm_status launch_rc) {
  bm_completion c{};
  c.id = sl.job.req.id;
  c.t_submit_us = sl.job.t_submit_us;
  c.fallback = sl.job.fallback;
  const int nrhs = sl.job.req.nrhs;
  const bool mixed = sl.job.precision == BM_PREC_FP32_IR;
  if (launch_rc != BM_OK) {
    c.status = launch_rc;
    c.t_start_us = c.t_factor_us = c.t_done_us = -1.0;
    for (int j = 0; j < nrhs; ++j) c.backward_error[j] = -1.0;
  } else {
    c.t_start_us = event_us(s, sl.ev_start);
    c.t_factor_us = event_us(s, sl.ev_factor);
    c.t_done_us = event_us(s, sl.ev_done);
    const Status &f = sl.hs[0];
    c.status = f.code;
    if (f.code == BM_ERR_NOT_SPD) {
      c.fail_scenario = f.scenario;
      c.fail_stage = f.stage;
    }
    for (int j = 0; j < nrhs; ++j) {
      const Status &v = sl.hs[1 + j];
      c.iters[j] = mixed ? v.iters : 0;
      c.backward_error[j] = mixed ? v.eta : -1.0;
      // the status word is sticky over the solves of one factor: rate each
      // right-hand side by its own backward error
      int code = v.code;
      if (mixed && code == BM_ERR_NOT_CONVERGED) code = v.eta <= s->desc.tol ? BM_OK : BM_ERR_NOT_CONVERGED;
      if (c.status == BM_OK && code != BM_OK) c.status = code;
    }
  }
  if (sl.h) release_impl(sl.h);
  sl.h = nullptr;
  s->arena->release(sl.off, sl.job.bytes);
  sl.busy = false;
  s->stats.in_flight--;
  if (sl.job.fallback) c.t_start_us = sl.job.t_first_start_us;
  // a mixed attempt that the FP32 tails could not resolve runs again in FP64
  IoLayout L64;
  if (mixed && (s->desc.flags & BM_SERVE_FP64_FALLBACK) && launch_rc == BM_OK &&
      (c.status == BM_ERR_NOT_SPD || c.status == BM_ERR_NOT_CONVERGED) &&
      layout_of(s->desc, BM_PREC_FP64, sl.job.req, &L64) && L64.total <= s->arena->capacity()) {
    Pending p = sl.job;
    p.precision = BM_PREC_FP64;
    p.fallback = 1;
    p.bytes = L64.total;
    p.t_first_start_us = c.t_start_us;
    s->queue.push_front(p);
    s->stats.queued++;
    s->stats.fallbacks++;
    return;
  }
  s->stats.completed++;
  s->done.push_back(c);
}

// One pass of the loop: retire finished requests, then admit from the head
// of the queue while a slot and memory are free.
static bm_status advance(bm_server s) {
  bm_status worst = BM_OK;
  for (Slot &sl : s->slots) {
    if (!sl.busy) continue;
    const cudaError_t e = cudaEventQuery(sl.ev_done);
    if (e == cudaErrorNotReady) continue;
    if (e != cudaSuccess) {
      cudaGetLastError();
      worst = BM_ERR_CUDA;
      retire(s, sl, BM_ERR_CUDA);
      continue;
    }
    retire(s, sl, BM_OK);
  }
  while (!s->queue.empty()) {
    Slot *free_slot = nullptr;
    for (Slot &sl : s->slots)
      if (!sl.busy) {
        free_slot = &sl;
        break;
      }
    if (!free_slot) break;
    Pending &head = s->queue.front();
    const size_t off = s->arena->alloc(head.bytes);
    if (off == SIZE_MAX) break;   // first in, first out: the head waits for memory
    Slot &sl = *free_slot;
    sl.job = head;
    sl.off = off;
    sl.busy = true;
    s->queue.pop_front();
    s->stats.queued--;
    s->stats.admitted++;
    s->stats.in_flight++;
    if (s->arena->used() > s->stats.peak_bytes_in_use) s->stats.peak_bytes_in_use = s->arena->used();
    const bm_status rc = launch_request(s, sl);
    if (rc != BM_OK) {
      // drain what was queued on the slot before handing its range back
      cudaStreamSynchronize(sl.stream);
      cudaGetLastError();
      retire(s, sl, rc);
      worst = rc;
    }
  }
  s->stats.bytes_in_use = s->arena->used();
  return worst;
}

extern "C" bm_status bm_server_submit(bm_server s, const bm_request *req) {
  if (!s || !valid_request(s->desc, req)) return BM_ERR_INVALID_ARG;
  IoLayout L;
  if (!layout_of(s->desc, s->desc.precision, *req, &L) || L.total > s->arena->capacity()) return BM_ERR_INVALID_ARG;
  Pending p{};
  p.req = *req;
  p.t_submit_us = now_us(s->t0);
  p.bytes = L.total;
  p.precision = s->desc.precision;
  s->queue.push_back(p);
  s->stats.submitted++;
  s->stats.queued++;
  advance(s);
  return BM_OK;
}

extern "C" bm_status bm_server_poll(bm_server s, int wait, bm_completion *out, int max_out, int *n_out) {
  if (!s || (max_out > 0 && !out)) return BM_ERR_INVALID_ARG;
  bm_status rc = advance(s);
  while (wait && s->done.empty() && (s->stats.in_flight > 0 || s->stats.queued > 0)) {
    // the oldest request in flight finishes first more often than not
    for (Slot &sl : s->slots)
      if (sl.busy) {
        cudaEventSynchronize(sl.ev_done);
        break;
      }
    const bm_status r2 = advance(s);
    if (rc == BM_OK) rc = r2;
  }
  int n = 0;
  while (n < max_out && !s->done.empty()) {
    out[n++] = s->done.front();
    s->done.pop_front();
  }
  if (n_out) *n_out = n;
  return rc;
}

extern "C" bm_status bm_server_get_stats(bm_server s, bm_server_stats *out) {
  if (!s || !out) return BM_ERR_INVALID_ARG;
  *out = s->stats;
  return BM_OK;
}

extern "C" void bm_server_destroy(bm_server s) {
  if (!s) return;
  free_server(s);
}
