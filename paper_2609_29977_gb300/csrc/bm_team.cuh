// Team-level building blocks for the tail kernels.
//
// A "team" is TEAM consecutive threads of a CTA that together process one
// task (one chain position of one tail). TEAM < 32 packs several teams into
// a warp: their single-lane steps (the pivot reciprocal square roots of the
// Cholesky) then execute in the same warp instruction, which matters on
// GB300 where the FP64 pipe charges a full warp instruction whatever the
// number of active lanes. TEAM >= 64 spreads one task over several warps
// (several SM sub-partitions) to shorten its dependent chains when a level
// has few tasks. Teams synchronize with __syncwarp(mask) or a named barrier.
//
// Blocks are NB x NB, row-major in shared memory with row stride NB; NB is a
// compile-time constant so every loop below has a static trip count.
#pragma once

#include <math.h>

#include "bm_internal.cuh"

namespace bm {

template <int TEAM>
struct Team {
  int lane, id;
  unsigned mask;
  __device__ __forceinline__ Team() {
    lane = threadIdx.x % TEAM;
    id = threadIdx.x / TEAM;
    if (TEAM < 32)
      mask = ((1u << (TEAM & 31)) - 1u) << ((threadIdx.x & 31) / TEAM * TEAM);
    else
      mask = 0xffffffffu;
  }
  __device__ __forceinline__ void sync() const {
    if (TEAM < 32)
      __syncwarp(mask);
    else if (TEAM == 32)
      __syncwarp();
    else
      asm volatile("bar.sync %0, %1;" ::"r"(id + 1), "r"(TEAM) : "memory");
  }
};

// Lower-triangle element e -> (i, j), j <= i (FP32 and integer ops only).
__device__ __forceinline__ void tri_index(int e, int &i, int &j) {
  int t = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
  t += ((t + 1) * (t + 2) / 2 <= e);
  t -= (t * (t + 1) / 2 > e);
  i = t;
  j = e - t * (t + 1) / 2;
}

template <typename T>
__device__ __forceinline__ T fma_t(T a, T b, T c);
template <>
__device__ __forceinline__ double fma_t<double>(double a, double b, double c) { return fma(a, b, c); }
template <>
__device__ __forceinline__ float fma_t<float>(float a, float b, float c) { return fmaf(a, b, c); }

template <typename T>
__device__ __forceinline__ T rsqrt_t(T x);
template <>
__device__ __forceinline__ double rsqrt_t<double>(double x) { return rsqrt(x); }
template <>
__device__ __forceinline__ float rsqrt_t<float>(float x) { return rsqrtf(x); }

// d > 0 and finite, tested on the bit pattern with integer instructions
// (positive IEEE values order like their bit patterns; NaN and -0 fail).
template <typename T>
__device__ __forceinline__ bool pivot_ok(T d);
template <>
__device__ __forceinline__ bool pivot_ok<double>(double d) {
  const long long b = __double_as_longlong(d);
  return b > 0ll && b < 0x7ff0000000000000ll;
}
template <>
__device__ __forceinline__ bool pivot_ok<float>(float d) {
  const int b = __float_as_int(d);
  return b > 0 && b < 0x7f800000;
}

// FP64 -> FP32 rounding to nearest even, done with integer instructions
// from the IEEE 754 binary64/binary32 encodings (on this GPU the F2F
// conversion instruction runs on the slow FP64 pipe). Overflow gives inf,
// results below the FP32 normal range are rounded to subnormals or zero,
// NaN stays NaN.
__device__ __forceinline__ float d2f_rn_slow(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ff);
  unsigned long long m = b & 0x000fffffffffffffull;
  if (e == 0x7ff) return __uint_as_float(sign | 0x7f800000u | (m ? 0x00400000u : 0u));
  const int e32 = e - 1023 + 127;
  if (e32 >= 255) return __uint_as_float(sign | 0x7f800000u);
  if (e32 <= 0) {
    const int shift = 1 - e32;
    if (e == 0 || shift > 24) return __uint_as_float(sign);
    m |= 1ull << 52;
    const int sh = 29 + shift;
    unsigned long long q = m >> sh;
    const unsigned long long rem = m & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (q & 1ull))) ++q;
    return __uint_as_float(sign | (unsigned)q);
  }
  const unsigned long long rem = m & ((1ull << 29) - 1), half = 1ull << 28;
  unsigned bits = ((unsigned)e32 << 23) | (unsigned)(m >> 29);
  if (rem > half || (rem == half && (bits & 1u))) ++bits;
  return __uint_as_float(sign | bits);
}

// Fast path with 32-bit integer instructions for results in the FP32 normal
// range (binary64 exponent 897..1150); everything else goes to d2f_rn_slow.
__device__ __forceinline__ float d2f_rn(double d) {
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  const unsigned e = (hi >> 20) & 0x7ffu;
  if (e - 897u < 253u) {
    unsigned bits = (hi & 0x80000000u) | ((e - 896u) << 23) | ((hi & 0x000fffffu) << 3) | (lo >> 29);
    const unsigned rem = lo & 0x1fffffffu;
    bits += (rem > 0x10000000u) | ((rem == 0x10000000u) & bits);
    return __uint_as_float(bits);
  }
  return d2f_rn_slow(d);
}

// FP32 -> FP64 (exact), with integer instructions.
__device__ __forceinline__ double f2d_exact(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned sign = b & 0x80000000u;
  int e = (int)((b >> 23) & 0xff);
  unsigned m = b & 0x007fffffu;
  if (e == 0xff) return __hiloint2double((int)(sign | 0x7ff00000u | (m >> 3)), (int)(m << 29));
  if (e == 0) {
    if (m == 0) return __hiloint2double((int)sign, 0);
    const int lz = __clz(m) - 8;   // bring the leading one to bit 23
    m = (m << lz) & 0x007fffffu;
    e = 1 - lz;
  }
  const unsigned ed = (unsigned)(e - 127 + 1023);
  return __hiloint2double((int)(sign | (ed << 20) | (m >> 3)), (int)(m << 29));
}

template <typename T>
__device__ __forceinline__ T to_t(double d);
template <>
__device__ __forceinline__ double to_t<double>(double d) { return d; }
template <>
__device__ __forceinline__ float to_t<float>(double d) { return d2f_rn(d); }

template <typename T>
__device__ __forceinline__ double to_d(T x);
template <>
__device__ __forceinline__ double to_d<double>(double x) { return x; }
template <>
__device__ __forceinline__ double to_d<float>(float x) { return f2d_exact(x); }

// Programmatic dependent launch: wait for the preceding kernel's results /
// let the next kernel start its launch. Both are no-ops without PDL.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <int TEAM, int N, typename T>
__device__ __forceinline__ void team_copy(const Team<TEAM> &tm, T *__restrict__ dst, const T *__restrict__ src) {
#pragma unroll
  for (int i = tm.lane; i < N; i += TEAM) dst[i] = src[i];
}
// dst (NB x NB) := src^T
template <int TEAM, int NB, typename T>
__device__ __forceinline__ void team_copy_t(const Team<TEAM> &tm, T *__restrict__ dst, const T *__restrict__ src) {
#pragma unroll
  for (int e = tm.lane; e < NB * NB; e += TEAM) {
    const int i = e / NB, j = e - i * NB;
    dst[j * NB + i] = src[e];
  }
}
template <int TEAM, int N, typename T>
__device__ __forceinline__ void team_zero(const Team<TEAM> &tm, T *dst) {
#pragma unroll
  for (int i = tm.lane; i < N; i += TEAM) dst[i] = T(0);
}
template <int TEAM, int NB, typename T>
__device__ __forceinline__ void team_store_lower(const Team<TEAM> &tm, T *__restrict__ g, const T *__restrict__ s) {
#pragma unroll
  for (int e = tm.lane; e < NB * NB; e += TEAM) {
    const int i = e / NB, j = e - i * NB;
    g[e] = (j <= i) ? s[e] : T(0);
  }
}

// Stores a diagonal factor block L (lower triangle of s, inverse diagonal
// in inv). For T = double the strict upper triangle of g receives the
// transpose of M = L diag(L)^-1, the unit lower triangular factor with
// columns scaled by the inverse pivots: g[i][j] = L_ji * inv_i for i < j.
// The tail solves then substitute with M and scale once (L y = z is
// M w = z, y = inv .* w; L^T x = z is M^T x = inv .* z), one FP64
// instruction per elimination step instead of two. For T = float the
// upper triangle is zero.
template <int TEAM, int NB, typename T>
__device__ __forceinline__ void team_store_factor(const Team<TEAM> &tm, T *__restrict__ g, const T *__restrict__ s,
                                                  const T *__restrict__ inv) {
#pragma unroll
  for (int e = tm.lane; e < NB * NB; e += TEAM) {
    const int i = e / NB, j = e - i * NB;
    T val = T(0);
    if (j <= i)
      val = s[e];
    else if (sizeof(T) == sizeof(double))
      val = s[j * NB + i] * inv[i];
    g[e] = val;
  }
}

// lower(sD) -= X X^T (+ Y Y^T when Y != null).
template <int TEAM, int NB, typename T>
__device__ __forceinline__ void team_syrk_sub(const Team<TEAM> &tm, T *sD, const T *X, const T *Y) {
  constexpr int NE = NB * (NB + 1) / 2;
#pragma unroll 1
  for (int e = tm.lane; e < NE; e += TEAM) {
    int i, j;
    tri_index(e, i, j);
    T acc = sD[i * NB + j];
#pragma unroll
    for (int k = 0; k < NB; ++k) acc = fma_t<T>(-X[i * NB + k], X[j * NB + k], acc);
    if (Y) {
#pragma unroll
      for (int k = 0; k < NB; ++k) acc = fma_t<T>(-Y[i * NB + k], Y[j * NB + k], acc);
    }
    sD[i * NB + j] = acc;
  }
}

// In-place lower Cholesky of sA; sInv[j] = 1/L_jj. A non-positive or
// non-finite pivot is replaced by 1; returns 1 + its column, 0 if none.
// Two barriers per column: the first element of each trailing update is
// the next diagonal entry, so its lane (lane 0) takes the next pivot step
// at once while the other lanes finish the update.
template <int TEAM, int NB, typename T>
__device__ __forceinline__ int team_chol(const Team<TEAM> &tm, T *sA, T *sInv) {
  int fail = 0;
  auto pivot = [&](int j, T d) {
    if (!pivot_ok(d)) {
      if (!fail) fail = j + 1;
      d = T(1);
    }
    const T r = rsqrt_t<T>(d);
    sA[j * NB + j] = d * r;
    sInv[j] = r;
  };
  if (tm.lane == 0) pivot(0, sA[0]);
  tm.sync();
#pragma unroll 1
  for (int j = 0; j < NB - 1; ++j) {
    const T r = sInv[j];
    for (int i = j + 1 + tm.lane; i < NB; i += TEAM) sA[i * NB + j] *= r;
    tm.sync();
    const int m = NB - 1 - j, ne = m * (m + 1) / 2;
    int e0 = tm.lane;
    if (tm.lane == 0) {   // element 0 of the trailing update is (j+1, j+1)
      const int d = (j + 1) * NB;
      pivot(j + 1, fma_t<T>(-sA[d + j], sA[d + j], sA[d + j + 1]));
      e0 = TEAM;
    }
    for (int e = e0; e < ne; e += TEAM) {
      int a, b;
      tri_index(e, a, b);
      const int i = j + 1 + a, k = j + 1 + b;
      sA[i * NB + k] = fma_t<T>(-sA[i * NB + j], sA[k * NB + j], sA[i * NB + k]);
    }
    tm.sync();
  }
  return fail;
}

// X (M x NB) := X L^{-T}, with the inverse diagonal of L in inv. One
// barrier per column: column j+1 is updated and scaled by inv[j+1] in the
// same pass (final for step j+1), then the columns after it are updated.
template <int TEAM, int NB, typename T>
__device__ __forceinline__ void team_trsm_lt(const Team<TEAM> &tm, T *X, int M, const T *L, const T *inv) {
  const T r0 = inv[0];
  for (int row = tm.lane; row < M; row += TEAM) X[row * NB] *= r0;
  tm.sync();
#pragma unroll 1
  for (int j = 0; j < NB - 1; ++j) {
    const T rn = inv[j + 1], l1 = L[(j + 1) * NB + j];
    for (int row = tm.lane; row < M; row += TEAM)
      X[row * NB + j + 1] = fma_t<T>(-X[row * NB + j], l1, X[row * NB + j + 1]) * rn;
    const int cols = NB - 2 - j, ne = M * cols;
    for (int e = tm.lane; e < ne; e += TEAM) {
      const int row = e / cols, k = j + 2 + (e - row * cols);
      X[row * NB + k] = fma_t<T>(-X[row * NB + j], L[k * NB + j], X[row * NB + k]);
    }
    tm.sync();
  }
}

// out (NB x NB, global) := -A B^T.
template <int TEAM, int NB, typename T>
__device__ __forceinline__ void team_gemm_nt_neg(const Team<TEAM> &tm, T *__restrict__ out, const T *A, const T *B) {
#pragma unroll 1
  for (int e = tm.lane; e < NB * NB; e += TEAM) {
    const int i = e / NB, j = e - i * NB;
    T acc = T(0);
#pragma unroll
    for (int k = 0; k < NB; ++k) acc = fma_t<T>(-A[i * NB + k], B[j * NB + k], acc);
    out[e] = acc;
  }
}

}  // namespace bm
