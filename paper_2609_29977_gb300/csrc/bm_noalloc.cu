// bm_factor_solve_noalloc: FP64 factor + solve that allocates no device
// memory.
//
// Some callers cannot call cudaMalloc: code that runs inside an allocator
// or memory-pool callback, real-time control loops whose certification
// forbids allocation after start-up, and hosts that hand this library a
// fixed device-memory budget and account for every byte. For them this
// entry point keeps every factor block and workspace of one system in a
// fixed array that the library itself defines below, instead of the
// handle-owned memory that bm_analyze allocates. The caller passes only
// the inputs (D, E, C, R, r) and the output x.
//
// The array is a file-scope __device__ variable of BM_NOALLOC_SCRATCH_BYTES
// bytes: every GPU that loads the library holds it until the process exits.
// In host code its name is only a host-side stand-in, so the first call on
// each device looks up its device address with cudaGetSymbolAddress (with
// that device current) and keeps it. Every call ends by copying the device
// status to the host and synchronizing the stream, so the entry point is
// synchronous and cannot be recorded into a CUDA graph: on a stream that is
// being captured it returns BM_ERR_INVALID_ARG before touching anything.
// All calls share the one array and it keeps the last call's contents, so
// the status word and the cross-CTA counters are cleared at the start of
// every call, and two calls whose work overlaps on the GPU (different
// streams, or different host threads) race on it.
#include <cuda_runtime.h>

#include <mutex>

#include "bm_internal.cuh"

namespace bm {
size_t f64_factor_smem(int nb, int nr);
cudaError_t f64_prepare(int nb, int nr);
void f64_launch_factor(const F64View &v, cudaStream_t st, const TailSched *sc = nullptr);
void f64_launch_solve(const F64View &v, const double *r, double *x, double *r0t, cudaStream_t st);
}  // namespace bm

using namespace bm;

static __device__ __align__(256) unsigned char g_noalloc_scratch[BM_NOALLOC_SCRATCH_BYTES];

namespace {

const int kMaxDevices = 64;
const size_t kStatusBytes = 512;   // Status at 0, last-block counters at 256
void *g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_setup_mutex;

size_t noalloc_bytes(int S, int N, int nb, int nr) {
  const size_t SN = (size_t)S * N, b2 = (size_t)nb * nb;
  size_t t = kStatusBytes;
  t += align_up(SN * b2 * sizeof(double), 256) * 5;          // Ld Ll Lr Dt W
  t += align_up((size_t)S * nr * nb * sizeof(double), 256);  // F
  t += align_up((size_t)S * nr * nr * sizeof(double), 256);  // U
  t += align_up((size_t)nr * nr * sizeof(double), 256) * 2;  // LR Rt
  t += align_up(SN * nb * sizeof(double), 256) * 3;          // invd y zt
  t += align_up((size_t)S * nr * sizeof(double), 256);       // tb
  t += align_up((size_t)nr * sizeof(double), 256);           // r0t
  return t;
}

// Device address of the scratch array on the current device (set up once).
bm_status scratch_on_current_device(void **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return BM_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return BM_ERR_CUDA;
    }
    if (f64_prepare(64, 64) != cudaSuccess) {
      cudaGetLastError();
      return BM_ERR_CUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return BM_OK;
}

}  // namespace

extern "C" bm_status bm_factor_solve_noalloc(int S, int N, int nb, int nr, const double *D, const double *E,
                                             const double *C, const double *R, const double *r, double *x,
                                             void *stream) {
  if (S < 1 || N < 1 || nb < 1 || nr < 1 || nb > 64 || nr > 64 || S > 65535) return BM_ERR_INVALID_ARG;
  if (!D || !C || !R || !r || !x || (N > 1 && !E) || (const void *)r == (const void *)x)
    return BM_ERR_INVALID_ARG;
  if (noalloc_bytes(S, N, nb, nr) > (size_t)BM_NOALLOC_SCRATCH_BYTES) return BM_ERR_INVALID_ARG;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing((cudaStream_t)stream, &cap) != cudaSuccess) {
    cudaGetLastError();
    return BM_ERR_CUDA;
  }
  if (cap != cudaStreamCaptureStatusNone) return BM_ERR_INVALID_ARG;
  void *base = nullptr;
  bm_status s = scratch_on_current_device(&base);
  if (s != BM_OK) return s;

  char *p = (char *)base + kStatusBytes;
  auto take = [&](size_t bytes) {
    double *q = (double *)p;
    p += align_up(bytes, 256);
    return q;
  };
  const size_t SN = (size_t)S * N, b2 = (size_t)nb * nb;
  F64View v{};
  v.S = S; v.N = N; v.nb = nb; v.nr = nr; v.Lc = chain_levels(N);
  v.D = D; v.E = E; v.C = C; v.R = R;
  v.Ld = take(SN * b2 * 8); v.Ll = take(SN * b2 * 8); v.Lr = take(SN * b2 * 8);
  v.Dt = take(SN * b2 * 8); v.W = take(SN * b2 * 8);
  v.F = take((size_t)S * nr * nb * 8); v.U = take((size_t)S * nr * nr * 8);
  v.LR = take((size_t)nr * nr * 8); v.Rt = take((size_t)nr * nr * 8);
  v.invd = take(SN * nb * 8); v.y = take(SN * nb * 8); v.zt = take(SN * nb * 8);
  v.tb = take((size_t)S * nr * 8);
  double *r0t = take((size_t)nr * 8);
  v.status = (Status *)base;
  v.tickets = (unsigned *)((char *)base + 256);

  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(base, 0, kStatusBytes, st) != cudaSuccess) {
    cudaGetLastError();
    return BM_ERR_CUDA;
  }
  f64_launch_factor(v, st);
  f64_launch_solve(v, r, x, r0t, st);
  if (cudaGetLastError() != cudaSuccess) return BM_ERR_CUDA;
  Status hs;
  if (cudaMemcpyAsync(&hs, base, sizeof(Status), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return BM_ERR_CUDA;
  }
  return (bm_status)hs.code;
}
