// Assembly front end (App. A, "Linear System Sparsity in IPM and ADMM"):
// the reduced SPD matrix K = P + tau I + delta^{-1} A^T A + G^T (W + delta I)^{-1} G
// of a branch-MPC QP, written straight into the block layout that
// bm_factor reads (D, E, C, R of Sec. III-B).
//
// Stage k = 1..N of scenario s holds z_k = (x_k, u_k) (nb = nx + nu); the
// root is u_0 (nr = nu). The equality rows are x_1 - B_0 u_0 (= A_0 x_init)
// and x_{k+1} - A_k x_k - B_k u_k (k = 1..N-1); G = I. Hence
//   D_k = diag(q_k, rw_k) + tau I + diag(1 / (w_k + delta))
//         + delta^{-1} ( [I 0; 0 0]                      (row defining x_k)
//                      + [A_k B_k]^T [A_k B_k] )          (k <= N-1)
//   E_k (block (k+1, k)) = -delta^{-1} [A_k B_k; 0 0]
//   C_s = -delta^{-1} [B_0^T 0]
//   R = diag(r0w) + tau I + diag(1 / (w0 + delta)) + delta^{-1} sum_s B_0^T B_0.
// The stage blocks are formed one CTA per stage (FP64 FMAs of A_k^T A_k are
// the bound), the coupling blocks one thread per entry, and each root entry
// by one CTA whose sum over scenarios has a fixed order, so no result
// depends on the launch shape.
#include <cuda_runtime.h>

#include <mutex>

#include "bm_internal.cuh"

namespace bm {
namespace {

struct QPView {
  int S, N, nx, nu;
  double tau, delta;
  const double *A, *B, *q, *rw, *r0w, *w, *w0;
  double *D, *E, *C, *R;
};

// One CTA per stage (s, k): [A_k B_k] (nx x nb) staged in shared memory,
// the lower triangle of [A_k B_k]^T [A_k B_k] computed once per pair and
// mirrored (FP64 FMAs are the bound: nx per pair), then D_k written whole
// and, for k <= N-1, E_k = -delta^{-1} [A_k B_k; 0 0] written from the
// staged block. Dynamic shared memory: (nx * nb + nb * nb) doubles.
__global__ void __launch_bounds__(256) k_assemble_stage(QPView v) {
  extern __shared__ double smem[];
  const int nx = v.nx, nu = v.nu, nb = nx + nu, N = v.N;
  double *M = smem, *T = smem + nx * nb;   // T[a * nb + b] = (M^T M)_{ab}, a >= b
  const double inv_d = 1.0 / v.delta;
  const long nblk = (long)v.S * N;
  for (long blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    const int s = (int)(blk / N), k = (int)(blk - (long)s * N) + 1;   // stage k, 1-based
    const bool dyn = k <= N - 1;                                     // row x_{k+1} - A_k x_k - B_k u_k
    const size_t sk = (size_t)s * N + k;                             // index of A_k, B_k
    __syncthreads();   // the previous stage's reads of M and T are done
    if (dyn) {
      for (int e = threadIdx.x; e < nx * nb; e += blockDim.x) {
        const int m = e / nb, c = e - m * nb;
        M[e] = c < nx ? v.A[(sk * nx + m) * nx + c] : v.B[(sk * nx + m) * nu + (c - nx)];
      }
    }
    __syncthreads();
    const int npair = nb * (nb + 1) / 2;
    for (int t = threadIdx.x; t < npair; t += blockDim.x) {
      int a = 0;
      while ((a + 1) * (a + 2) / 2 <= t) ++a;
      const int c = t - a * (a + 1) / 2;   // pair (a, c), c <= a
      double acc = 0.0;
      if (dyn)
        for (int m = 0; m < nx; ++m) acc = fma(M[m * nb + a], M[m * nb + c], acc);
      if (a == c && a < nx) acc += 1.0;    // the row that defines x_k
      double val = acc * inv_d;
      if (a == c) {
        const size_t sv = (size_t)s * N + (k - 1);
        const double p = a < nx ? v.q[sv * nx + a] : v.rw[sv * nu + (a - nx)];
        val += p + v.tau + 1.0 / (v.w[sv * nb + a] + v.delta);
      }
      T[a * nb + c] = val;
    }
    __syncthreads();
    double *Dk = v.D + (size_t)blk * nb * nb;
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
      const int i = e / nb, j = e - i * nb;
      Dk[e] = i >= j ? T[i * nb + j] : T[j * nb + i];
    }
    if (dyn) {
      double *Ek = v.E + ((size_t)s * (N - 1) + (k - 1)) * nb * nb;   // block (k+1, k)
      for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        const int i = e / nb;
        Ek[e] = i < nx ? -M[e] * inv_d : 0.0;   // row i of [A_k B_k] is M[i * nb ...]
      }
    }
  }
}

// C_s = -delta^{-1} [B_0^T 0], one thread per entry.
__global__ void k_assemble_coupling(QPView v) {
  const int nx = v.nx, nu = v.nu, nb = nx + nu;
  const long nC = (long)v.S * nu * nb;
  const double inv_d = 1.0 / v.delta;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < nC; e += (long)gridDim.x * blockDim.x) {
    const int s = (int)(e / (nu * nb));
    const int cj = (int)(e - (long)s * nu * nb), c = cj / nb, j = cj - c * nb;
    v.C[e] = j < nx ? -v.B[((size_t)s * v.N * nx + j) * nu + c] * inv_d : 0.0;   // B_0 of scenario s
  }
}

// R, one CTA of 256 threads per entry (a, b): thread t sums the scenarios
// s = t, t + 256, ... in increasing s, then a fixed shared-memory tree adds
// the 256 partial sums (the same order for every launch).
__global__ void __launch_bounds__(256) k_assemble_root(QPView v) {
  __shared__ double red[256];
  const int nx = v.nx, nu = v.nu;
  const int a = blockIdx.x / nu, b = blockIdx.x - a * nu;
  double acc = 0.0;
  for (int s = threadIdx.x; s < v.S; s += blockDim.x) {
    const double *B0 = v.B + (size_t)s * v.N * nx * nu;
    for (int m = 0; m < nx; ++m) acc = fma(B0[m * nu + a], B0[m * nu + b], acc);
  }
  red[threadIdx.x] = acc;
  for (int h = blockDim.x >> 1; h > 0; h >>= 1) {
    __syncthreads();
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
  }
  if (threadIdx.x == 0) {
    double val = red[0] / v.delta;
    if (a == b) val += v.r0w[a] + v.tau + 1.0 / (v.w0[a] + v.delta);
    v.R[blockIdx.x] = val;
  }
}

}  // namespace
}  // namespace bm

using namespace bm;

extern "C" bm_status bm_assemble_reduced(const bm_qp_desc *d, const double *A, const double *B, const double *q,
                                         const double *rw, const double *r0w, const double *w, const double *w0,
                                         double *D, double *E, double *C, double *R, void *stream) {
  if (!d || d->S < 1 || d->N < 1 || d->nx < 1 || d->nu < 1 || d->nx + d->nu > 64 || d->nu > 64 || d->S > 65535)
    return BM_ERR_INVALID_ARG;
  if (!(d->tau >= 0.0) || !(d->delta > 0.0)) return BM_ERR_INVALID_ARG;
  if (!A || !B || !q || !rw || !r0w || !w || !w0 || !D || !C || !R || (d->N > 1 && !E)) return BM_ERR_INVALID_ARG;
  QPView v{d->S, d->N, d->nx, d->nu, d->tau, d->delta, A, B, q, rw, r0w, w, w0, D, E, C, R};
  cudaStream_t st = (cudaStream_t)stream;
  const int nb = d->nx + d->nu;
  const size_t smem = ((size_t)d->nx * nb + (size_t)nb * nb) * sizeof(double);
  static std::mutex attr_mu;
  static bool attr_set[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> attr_lock(attr_mu);
  if (dev >= 0 && dev < 64 && !attr_set[dev]) {
    // the largest block (nb = 64, nx = 63) needs 64 KB of dynamic shared memory
    if (cudaFuncSetAttribute(k_assemble_stage, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024) !=
        cudaSuccess)
      return BM_ERR_CUDA;
    attr_set[dev] = true;
  }
  long blocks = (long)d->S * d->N;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_assemble_stage<<<(unsigned)blocks, 256, smem, st>>>(v);
  const long cwork = (long)d->S * d->nu * nb;
  long cblocks = (cwork + 255) / 256;
  if (cblocks > 152 * 4) cblocks = 152 * 4;
  k_assemble_coupling<<<(unsigned)cblocks, 256, 0, st>>>(v);
  k_assemble_root<<<(unsigned)(d->nu * d->nu), 256, 0, st>>>(v);
  return cudaGetLastError() == cudaSuccess ? BM_OK : BM_ERR_CUDA;
}
