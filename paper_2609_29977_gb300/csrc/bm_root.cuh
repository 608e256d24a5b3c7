// The root step of the factor (Alg. 1 steps 4-5) as device routines shared
// by the FP64 root kernel and the per-tail top kernel that can finish it:
// R~ = R - sum_i U_i entry by entry (one warp per entry, the library's
// fixed summation order root_sum_warp) and L_R = chol(R~) by one CTA.
#pragma once

#include <math.h>

#include "bm_internal.cuh"

namespace bm {

// global (n x n) := lower triangle of s, zeros above
__device__ __forceinline__ void cta_store_lower(double *__restrict__ g, const double *__restrict__ s, int n) {
  const int n2 = n * n;
  for (int e = threadIdx.x; e < n2; e += blockDim.x) {
    const int i = e / n, j = e - i * n;
    g[e] = (j <= i) ? s[e] : 0.0;
  }
}

// Lower-triangle element e -> (i, j) with j <= i.
__device__ __forceinline__ void tri_ij(int e, int &i, int &j) {
  int t = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
  while ((t + 1) * (t + 2) / 2 <= e) ++t;
  while (t * (t + 1) / 2 > e) --t;
  i = t;
  j = e - t * (t + 1) / 2;
}

// In-place lower Cholesky of the n x n block sA (lower triangle read);
// sInv[j] = 1 / L_jj. A pivot that is not positive and finite is replaced by
// 1 (so the launch finishes without NaNs) and the first such column + 1 is
// returned; 0 on success.
__device__ inline int cta_chol(double *sA, double *sInv, int n, int *sflag) {
  if (threadIdx.x == 0) *sflag = 0;
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      double d = sA[j * n + j];
      if (!(d > 0.0) || !(d < INFINITY)) {
        if (*sflag == 0) *sflag = j + 1;
        d = 1.0;
      }
      const double r = rsqrt(d);
      sA[j * n + j] = d * r;
      sInv[j] = r;
    }
    __syncthreads();
    const double r = sInv[j];
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) sA[i * n + j] *= r;
    __syncthreads();
    const int m = n - j - 1, ne = m * (m + 1) / 2;
    for (int e = threadIdx.x; e < ne; e += blockDim.x) {
      int a, b;
      tri_ij(e, a, b);
      const int i = j + 1 + a, k = j + 1 + b;
      sA[i * n + k] = fma(-sA[i * n + j], sA[k * n + j], sA[i * n + k]);
    }
    __syncthreads();
  }
  return *sflag;
}

// Entry e of the lower triangle of R~ = R - sum_i U_i, by one warp (all 32
// lanes), into Rt (both triangles).
__device__ __forceinline__ void root_entry(const double *U, const double *R, int S, int nr, int e, double *Rt) {
  int i, j;
  tri_ij(e, i, j);
  const double val = R[i * nr + j] - root_sum_warp(U, S, nr, i, j);
  if ((threadIdx.x & 31) == 0) {
    Rt[i * nr + j] = val;
    Rt[j * nr + i] = val;
  }
}

// L_R = chol(sR) (nr x nr in shared memory, followed by nr doubles of
// scratch) stored lower into LR. A failed pivot is reported at the root
// unless *engage (the mixed path's probe) takes over: then *on = engage
// and no failure is reported. Call with every thread of the CTA.
__device__ __forceinline__ void root_chol_store(double *sR, int nr, double *LR, Status *status, bool *engage,
                                                int *on) {
  __shared__ int sflag;
  const int fail = cta_chol(sR, sR + nr * nr, nr, &sflag);
  bool eng = false;
  if (engage) eng = *engage || fail;
  if (threadIdx.x == 0) {
    if (engage) *on = eng ? 1 : 0;
    if (fail && !eng) report_not_spd(status, -1, 0);
  }
  cta_store_lower(LR, sR, nr);
}

// The whole root step by one CTA: every entry (warps in turn), then the
// Cholesky. sm: nr * nr + nr doubles of shared memory.
__device__ __forceinline__ void root_reduce_chol(const double *U, const double *R, int S, int nr, double *Rt,
                                                 double *LR, Status *status, double *sm) {
  const int ne = nr * (nr + 1) / 2, nw = blockDim.x >> 5;
  for (int e = threadIdx.x >> 5; e < ne; e += nw) root_entry(U, R, S, nr, e, Rt);
  __threadfence_block();
  __syncthreads();
  for (int k = threadIdx.x; k < nr * nr; k += blockDim.x) sm[k] = Rt[k];
  __syncthreads();
  root_chol_store(sm, nr, LR, status, nullptr, nullptr);
}

}  // namespace bm
