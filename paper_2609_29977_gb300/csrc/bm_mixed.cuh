// Mixed-precision solve state and the device bodies shared by the single
// system kernels (bm_mixed.cu) and the batched kernels (bm_batch.cu).
#pragma once

#include "bm_ff.cuh"
#include "bm_tail_factor.cuh"

namespace bm {

struct IRCtl {
  int converged;            // stop flag: the stopping test held, or refinement stalled
  int iters;                // corrections applied in the last solve
  unsigned wmax;            // max_i omega_i of the running iteration (bits of a non-negative float)
  int loop;                 // index of the next iteration (read by the kernels of a graph loop body)
  double omega_prev;        // omega after the previous iteration
  double eta;               // omega after the last iteration
  int retry;                // automatic mode: this solve refines the coupling columns and continues
};

struct MixedState {
  int S, N, nb, nr, Lc;
  float *Ld, *Ll, *Lr, *Dt, *W, *invd;   // FP32 tail factor and level workspace
  double *F, *U, *LR, *Rt;               // FP64 root parts
  float *y, *zt;                         // [S][N][nb] solve vectors (y is overwritten by the correction)
  double *tb;                            // [S][nr] per-tail root terms (with refined coupling columns: [grid][nr] per-CTA parts)
  double *d0;                            // [nr] root correction
  // refined coupling columns X_i = K_i^{-1} C_i^T ([S][N][nb][ldc], FP32;
  // bm_coupling.cuh), used by the solve when *cxon is set; null when the
  // handle never refines them
  const float *Xc;
  int ldc;
  const int *cxon;
  int cmode;                             // 0: FP32-based root, 1: automatic, 2: always refine
  float *Xa, *Yb, *Zr;                   // coupling refinement buffers (Xa = Xc)
  double *rho;                           // [n] residual
  // float-float refinement residual (ffres = 1; else FP64): K split into
  // hi + lo floats once per factor (Kd: D as full symmetric rows
  // [S][N][nb][nb]; Ke: E as stored), the iterate x split by the backward
  // kernel ([S][N][nb])
  int ffres;
  float *Kdh, *Kdl, *Keh, *Kel, *xh, *xl;
  IRCtl *ctl;
  Status *status;
  unsigned *tickets;
  const double *D, *E, *C, *R;           // inputs of the last factor
};

namespace mx {

__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}
// |x| rounded down to FP32, from the bit pattern with integer instructions
// (for the row sums of |K|; only used for the norm in the stopping test).
__device__ __forceinline__ float abs_f32_approx(double x) {
  const unsigned hi = (unsigned)(__double_as_longlong(x) >> 32) & 0x7fffffffu;
  const int e = (int)(hi >> 20) - 1023 + 127;
  if (e <= 0) return 0.0f;
  if (e >= 255) return __uint_as_float(0x7f7fffffu);
  return __uint_as_float(((unsigned)e << 23) | ((hi & 0xfffffu) << 3));
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

template <int NB>
struct MCfg {
  static constexpr int TS = NB <= 4 ? 4 : NB <= 8 ? 8 : NB <= 16 ? 16 : NB <= 32 ? 32 : 64;
  static constexpr int THREADS = 256;
  static constexpr int TEAMS = THREADS / TS;
};

__device__ __forceinline__ bool ir_done(const IRCtl *ctl) {
  return *((volatile const int *)&ctl->converged) != 0;
}

// The iteration a kernel runs: its launch argument, or (iter < 0, inside the
// body of a graph loop) the counter the previous iteration's stopping test left.
__device__ __forceinline__ int ir_iter(const IRCtl *ctl, int iter) {
  return iter >= 0 ? iter : *((volatile const int *)&ctl->loop);
}

// z - sum_k L[k] y[k] over one row of a tail block (row-major, contiguous)
// and a vector written by other CTAs (read through L2), k in increasing
// order; four entries per load when the rows are 16-byte aligned.
template <int NB>
__device__ __forceinline__ float row_dot_sub(const float *__restrict__ L, const float *y, float z) {
  if constexpr (NB % 4 == 0) {
    const float4 *L4 = reinterpret_cast<const float4 *>(L);
    const float4 *y4 = reinterpret_cast<const float4 *>(y);
#pragma unroll
    for (int g = 0; g < NB / 4; ++g) {
      const float4 l = L4[g], v = __ldcg(y4 + g);
      z = fmaf(-l.x, v.x, z);
      z = fmaf(-l.y, v.y, z);
      z = fmaf(-l.z, v.z, z);
      z = fmaf(-l.w, v.w, z);
    }
  } else {
#pragma unroll
    for (int k = 0; k < NB; ++k) z = fmaf(-L[k], __ldcg(y + k), z);
  }
  return z;
}

// The same with the column of a block (L[k * NB], coalesced over the team)
// and the vector read four entries per load.
template <int NB>
__device__ __forceinline__ float col_dot_sub(const float *__restrict__ L, const float *y, float z) {
  if constexpr (NB % 4 == 0) {
    const float4 *y4 = reinterpret_cast<const float4 *>(y);
#pragma unroll
    for (int g = 0; g < NB / 4; ++g) {
      const float4 v = __ldcg(y4 + g);
      z = fmaf(-L[(4 * g) * NB], v.x, z);
      z = fmaf(-L[(4 * g + 1) * NB], v.y, z);
      z = fmaf(-L[(4 * g + 2) * NB], v.z, z);
      z = fmaf(-L[(4 * g + 3) * NB], v.w, z);
    }
  } else {
#pragma unroll
    for (int k = 0; k < NB; ++k) z = fmaf(-L[k * NB], __ldcg(y + k), z);
  }
  return z;
}

// One contiguous row of a block into registers (four floats per load when aligned).
template <int NB>
__device__ __forceinline__ void load_row(float (&r)[NB], const float *__restrict__ p) {
  if constexpr (NB % 4 == 0) {
    const float4 *p4 = reinterpret_cast<const float4 *>(p);
#pragma unroll
    for (int g = 0; g < NB / 4; ++g) {
      const float4 v = p4[g];
      r[4 * g] = v.x;
      r[4 * g + 1] = v.y;
      r[4 * g + 2] = v.z;
      r[4 * g + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < NB; ++k) r[k] = p[k];
  }
}

// The solve uses the refined coupling columns (bm_coupling.cuh).
__device__ __forceinline__ bool coupled(const MixedState &m) {
  return m.Xc != nullptr && *((volatile const int *)m.cxon) != 0;
}

// Fixed-order CTA sum of eight float-float values per thread (blockDim a
// multiple of 32, at most 256): a warp butterfly, then the warps in order;
// thread c < count writes the double hi + lo of sum c to out[c]. Call with
// every thread of the CTA.
__device__ __forceinline__ void ff_cta_sum8(float (&h)[8], float (&l)[8], double *out, int count) {
  __shared__ float sph[8][8], spl[8][8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const float hh = __shfl_xor_sync(0xffffffffu, h[c], o), ll = __shfl_xor_sync(0xffffffffu, l[c], o);
      float e;
      ff::two_sum(h[c], hh, h[c], e);
      l[c] = __fadd_rn(l[c], __fadd_rn(ll, e));
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      sph[warp][c] = h[c];
      spl[warp][c] = l[c];
    }
  }
  __syncthreads();
  if ((int)threadIdx.x < count && threadIdx.x < 8) {
    const int c = threadIdx.x;
    float hs = sph[0][c], ls = spl[0][c];
    for (int w = 1; w < nw; ++w) {
      float e;
      ff::two_sum(hs, sph[w][c], hs, e);
      ls = __fadd_rn(ls, __fadd_rn(spl[w][c], e));
    }
    out[c] = ff::to_double(hs, ls);
  }
  __syncthreads();
}

// Root terms with refined coupling columns: X^T v over the rows of all
// tails that this thread visits in a grid-stride walk (row e = blockIdx.x *
// blockDim.x + threadIdx.x + k * gridDim.x * blockDim.x), each product in
// a Dot2 sum (v split into hi + lo floats, X exactly FP32), combined per CTA
// by ff_cta_sum8 into tb[blockIdx.x][0..nr). The root step needs only the
// sum over all rows, so the grid's partials can mix tails; the fixed walk
// and reductions keep the bits independent of timing.
__device__ __forceinline__ void xt_grid(const MixedState &m, const double *__restrict__ v, int NBr) {
  const long nrow = (long)m.S * m.N * NBr;
  const long stride = (long)gridDim.x * blockDim.x;
  for (int c0 = 0; c0 < m.nr; c0 += 8) {
    float h[8], l[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) h[c] = l[c] = 0.0f;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < nrow; e += stride) {
      float vh, vl;
      ff::split_d(v[e], vh, vl);
      const float *xr = m.Xc + (size_t)e * m.ldc + c0;
      const float4 a = __ldg(reinterpret_cast<const float4 *>(xr));
      const float4 b = __ldg(reinterpret_cast<const float4 *>(xr + 4));
      const float xv[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
      for (int c = 0; c < 8; ++c) ff::dot2_step_split(h[c], l[c], vh, vl, xv[c]);
    }
    const int cnt = m.nr - c0 < 8 ? m.nr - c0 : 8;
    ff_cta_sum8(h, l, m.tb + (size_t)blockIdx.x * m.nr + c0, cnt);
  }
}

// Forward substitution of one tail in FP32 (all levels, then x_1 and
// t_i = F_{i,1} y_1 in FP64); the last CTA of the grid does the root step
// of Alg. 2 in FP64 and stores the root correction d_0 (and x_0 += d_0).
template <int NB>
__device__ __forceinline__ void fwd_tail(const MixedState &m, const double *__restrict__ rhs, int s, int crank,
                                         int CS, float (*sY)[NB]) {
  constexpr int TS = MCfg<NB>::TS, TEAMS = MCfg<NB>::TEAMS, NB2 = NB * NB;
  const Team<TS> tm;
  const int N = m.N, Lc = m.Lc;
  const size_t sb = (size_t)s * N;
  const int i = tm.lane;
  const bool xmode = coupled(m);
  for (int lvl = 0; lvl <= Lc; ++lvl) {
    const bool lastlvl = lvl == Lc;
    const int ntask = lastlvl ? 1 : (lvl == 0 ? N / 2 : ((N - 1) >> lvl) + 1);
    for (int t = crank * TEAMS + tm.id; t < ntask; t += CS * TEAMS) {
      int q;
      if (lastlvl) q = N;
      else if (lvl == 0) q = 2 * t + 1;
      else {
        const int cnt = (N - 1) >> lvl;
        q = t < cnt ? (t + 1) << lvl : N;
      }
      const bool elim = lastlvl || (q < N && ctz32(q) == lvl);
      const size_t zoff = (sb + (N - q)) * NB;
      // row i of L_qq and 1/L_ii: for NB <= 16 loaded first, so that they
      // share the gather's memory round trip (in bounds for every q); for
      // larger blocks after it (loaded first they slowed the nb = 48 solve)
      constexpr bool kEarly = NB <= 16;
      float Lrow[NB];
      float inv = 0.0f;
      if constexpr (kEarly) {
        load_row<NB>(Lrow, m.Ld + (sb + (N - q)) * NB2 + (i < NB ? i : 0) * NB);
        inv = i < NB ? m.invd[zoff + i] : 0.0f;
      }
      float z = 0.0f;
      if (i < NB) {
        z = (lvl <= 1) ? __double2float_rn(rhs[zoff + i]) : __ldcg(m.zt + zoff + i);
        if (lvl >= 1) {
          const int h = 1 << (lvl - 1);
          int pl = 0, pr = 0;
          if (q < N) {
            pl = q - h;
            if (q + h <= N - 1) pr = q + h;
          } else {
            const int mm = ((N - 1) >> (lvl - 1)) << (lvl - 1);
            if (ctz32(mm) == lvl - 1) pl = mm;
          }
          if (pl) z = row_dot_sub<NB>(m.Lr + (sb + (N - pl)) * NB2 + i * NB, m.y + (sb + (N - pl)) * NB, z);
          if (pr) z = row_dot_sub<NB>(m.Ll + (sb + (N - pr)) * NB2 + i * NB, m.y + (sb + (N - pr)) * NB, z);
        }
      }
      if (!elim) {
        if (i < NB) m.zt[zoff + i] = z;
        continue;
      }
      if constexpr (!kEarly) {
        load_row<NB>(Lrow, m.Ld + (sb + (N - q)) * NB2 + (i < NB ? i : 0) * NB);
        inv = i < NB ? m.invd[zoff + i] : 0.0f;
      }
      if (TS <= 32) {
        const int base = (threadIdx.x & 31) & ~(TS - 1);
#pragma unroll
        for (int j = 0; j < NB; ++j) {
          if (i == j) z *= inv;
          const float yj = __shfl_sync(tm.mask, z, base + j);
          if (i > j && i < NB) z = fmaf(-Lrow[j], yj, z);
        }
        if (i < NB) sY[tm.id][i] = z;
        tm.sync();
      } else {
#pragma unroll
        for (int j = 0; j < NB; ++j) {
          if (i == j) {
            z *= inv;
            sY[tm.id][j] = z;
          }
          tm.sync();
          if (i > j && i < NB) z = fmaf(-Lrow[j], sY[tm.id][j], z);
        }
      }
      if (i < NB) m.y[zoff + i] = z;
      if (lastlvl && !xmode) {
        tm.sync();
        const int nr = m.nr;
        const double *Fs = m.F + (size_t)s * nr * NB;
        for (int c = i; c < nr; c += TS) {
          double acc = 0.0;
#pragma unroll
          for (int k = 0; k < NB; ++k) acc = fma(Fs[c * NB + k], f2d_exact(sY[tm.id][k]), acc);
          m.tb[(size_t)s * nr + c] = acc;
        }
      }
      tm.sync();
    }
    if (CS > 1)
      cluster_sync();
    else
      __syncthreads();
  }
}

// Root step of Alg. 2 for one system, by one CTA once every tail's root
// term is in tb (t_i = F_{i,1} y_1, or with refined coupling columns the
// per-CTA parts of X_i^T rhs_i; nt entries): r~_0 = rhs_0 - sum_t tb_t,
// d_0 = L_R^{-T} L_R^{-1} r~_0 (FP64), x_0 += d_0. The sum over t is fixed
// in order: lane l of a warp adds the entries t = l, l + 32, ... in
// increasing t, and the 32 partial sums are combined by a fixed butterfly.
template <int NB>
__device__ __forceinline__ void root_step(const MixedState &m, const double *__restrict__ rhs, double *x, int iter,
                                          double *sR, int nt) {
  const int N = m.N, nr = m.nr, S = m.S;
  const size_t n0 = (size_t)S * N * NB;
  double *sL = sR, *sz = sR + nr * nr;
  for (int e = threadIdx.x; e < nr * nr; e += blockDim.x) sL[e] = __ldcg(m.LR + e);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int c = warp; c < nr; c += nw) {
    double acc = 0.0;
    for (int t = lane; t < nt; t += 32) acc += __ldcg(m.tb + (size_t)t * nr + c);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) sz[c] = rhs[n0 + c] - acc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int j = 0; j < nr; ++j) {
      double v = sz[j];
      for (int k = 0; k < j; ++k) v = fma(-sL[j * nr + k], sz[k], v);
      sz[j] = v / sL[j * nr + j];
    }
    for (int j = nr - 1; j >= 0; --j) {
      double v = sz[j];
      for (int k = j + 1; k < nr; ++k) v = fma(-sL[k * nr + j], sz[k], v);
      sz[j] = v / sL[j * nr + j];
    }
    for (int j = 0; j < nr; ++j) {
      m.d0[j] = sz[j];
      x[n0 + j] = (iter == 0 ? 0.0 : x[n0 + j]) + sz[j];
    }
  }
}

// Last-CTA election over n participating CTAs with the counter *ticket
// (reset by the winner). Call with all threads of the CTA.
__device__ __forceinline__ bool last_cta(unsigned *ticket, unsigned n) {
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    last = atomicAdd(ticket, 1u) == n - 1;
    if (last) *ticket = 0u;
  }
  __syncthreads();
  if (last) __threadfence();
  return last != 0;
}

// Backward substitution in FP32 fused with x += d (FP64); the correction of
// each position overwrites its forward vector y.
template <int NB>
__device__ __forceinline__ void bwd_tail(const MixedState &m, double *x, int iter, int s, int crank, int CS,
                                         float (*sX)[NB]) {
  constexpr int TS = MCfg<NB>::TS, TEAMS = MCfg<NB>::TEAMS, NB2 = NB * NB;
  const Team<TS> tm;
  const int N = m.N, Lc = m.Lc, nr = m.nr;
  const size_t sb = (size_t)s * N;
  const int i = tm.lane;
  const bool xmode = coupled(m);
  // d_0 as hi + lo floats for the tails' X_i d_0 (refined coupling columns)
  __shared__ float sdh[64], sdl[64];
  if (xmode) {
    for (int c = threadIdx.x; c < nr; c += blockDim.x) ff::split_d(__ldcg(m.d0 + c), sdh[c], sdl[c]);
    __syncthreads();
  }
  for (int lvl = Lc; lvl >= 0; --lvl) {
    const bool first = lvl == Lc;
    const int ntask = first ? 1 : (((N - 1) >> lvl) + 1) / 2;
    for (int t = crank * TEAMS + tm.id; t < ntask; t += CS * TEAMS) {
      const int q = first ? N : (2 * t + 1) << lvl;
      const size_t zoff = (sb + (N - q)) * NB;
      // column i of L_qq and 1/L_ii: loaded with the gather's operands for
      // NB <= 16, after the gather for larger blocks
      constexpr bool kEarly = NB <= 16;
      float Lcol[NB];
      float inv = 0.0f;
      if constexpr (kEarly) {
        const float *Ld = m.Ld + (sb + (N - q)) * NB2 + (i < NB ? i : 0);
#pragma unroll
        for (int k = 0; k < NB; ++k) Lcol[k] = Ld[k * NB];
        inv = i < NB ? m.invd[zoff + i] : 0.0f;
      }
      float z = 0.0f;
      if (i < NB) {
        if (first && xmode) {
          z = m.y[zoff + i];
        } else if (first) {
          double zd = f2d_exact(m.y[zoff + i]);
          const double *Fs = m.F + (size_t)s * nr * NB;
          for (int c = 0; c < nr; ++c) zd = fma(-Fs[c * NB + i], __ldcg(m.d0 + c), zd);
          z = __double2float_rn(zd);
        } else {
          z = m.y[zoff + i];
          const int h = 1 << lvl;
          const int a = q - h, b = (q + h <= N - 1) ? q + h : N;
          z = col_dot_sub<NB>(m.Lr + (sb + (N - q)) * NB2 + i, m.y + (sb + (N - b)) * NB, z);
          if (q > h) z = col_dot_sub<NB>(m.Ll + (sb + (N - q)) * NB2 + i, m.y + (sb + (N - a)) * NB, z);
        }
      }
      if constexpr (!kEarly) {
        const float *Ld = m.Ld + (sb + (N - q)) * NB2 + (i < NB ? i : 0);
#pragma unroll
        for (int k = 0; k < NB; ++k) Lcol[k] = Ld[k * NB];
        inv = i < NB ? m.invd[zoff + i] : 0.0f;
      }
      if (TS <= 32) {
        const int base = (threadIdx.x & 31) & ~(TS - 1);
#pragma unroll
        for (int j = NB - 1; j >= 0; --j) {
          if (i == j) z *= inv;
          const float xj = __shfl_sync(tm.mask, z, base + j);
          if (i < j) z = fmaf(-Lcol[j], xj, z);
        }
      } else {
#pragma unroll
        for (int j = NB - 1; j >= 0; --j) {
          if (i == j) {
            z *= inv;
            sX[tm.id][j] = z;
          }
          tm.sync();
          if (i < j) z = fmaf(-Lcol[j], sX[tm.id][j], z);
        }
      }
      if (i < NB) {
        m.y[zoff + i] = z;
        double dz;
        if (xmode) {
          // d_i = z - X_i d_0 on this row, the product summed by Dot2
          const float *xr = m.Xc + (zoff + i) * m.ldc;
          float h = 0.0f, l = 0.0f;
          for (int c = 0; c < nr; ++c) ff::dot2_step_split(h, l, sdh[c], sdl[c], __ldcg(xr + c));
          float dh, e;
          ff::two_sum(z, -h, dh, e);
          dz = ff::to_double(dh, __fsub_rn(e, l));
        } else {
          dz = f2d_exact(z);
        }
        const double xv = iter == 0 ? dz : x[zoff + i] + dz;
        x[zoff + i] = xv;
        if (m.ffres) {
          float h, l;
          ff::split_d(xv, h, l);
          m.xh[zoff + i] = h;
          m.xl[zoff + i] = l;
          if (ff::out_of_range(xv)) m.status->ffbad = 1;
        }
      }
      tm.sync();
    }
    if (CS > 1)
      cluster_sync();
    else
      __syncthreads();
  }
}



// Componentwise backward error (Oettli-Prager) of the refinement iterate:
// omega = max_i |r - K x|_i / (|K| |x| + |r|)_i. The residual itself is
// FP64; the weights |K||x| + |r| only scale it, so they are accumulated in
// FP32 from magnitudes rounded toward zero with integer instructions (the
// FP64 pipe stays free for the residual), which can only overstate omega.
__device__ __forceinline__ float omega_of(double rho, float w) {
  const float num = abs_f32_approx(rho);
  if (!(w > 0.0f)) return num == 0.0f ? 0.0f : __int_as_float(0x7f800000);
  return num / w;
}

// Row i of block row (s, k) of the residual: rho_i = r_i - (K x)_i (stored
// in m.rho) and its omega_i. Lanes i >= NB must not call it.
template <int NB>
__device__ __forceinline__ float residual_row(const MixedState &m, const double *__restrict__ r,
                                              const double *__restrict__ x, int s, int k, int i) {
  constexpr int NB2 = NB * NB;
  const int N = m.N, nr = m.nr;
  const size_t n0 = (size_t)m.S * N * NB;
  const long br = (long)s * N + k;
  const size_t off = (size_t)br * NB;
  const double *Dk = m.D + (size_t)br * NB2;
  const double *xk = x + off;
  const double ri = r[off + i];
  double acc = ri;
  float w = abs_f32_approx(ri);
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    const double kij = j <= i ? Dk[i * NB + j] : Dk[j * NB + i];
    const double xj = xk[j];
    acc = fma(-kij, xj, acc);
    w = fmaf(abs_f32_approx(kij), abs_f32_approx(xj), w);
  }
  if (k > 0) {   // block (k, k-1) = E_k (1-based stage k+1)
    const double *Ek = m.E + ((size_t)s * (N - 1) + (k - 1)) * NB2 + i * NB;
    const double *xp = xk - NB;
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      acc = fma(-Ek[j], xp[j], acc);
      w = fmaf(abs_f32_approx(Ek[j]), abs_f32_approx(xp[j]), w);
    }
  }
  if (k + 1 < N) {   // block (k, k+1) = E_{k+1}^T
    const double *Ek = m.E + ((size_t)s * (N - 1) + k) * NB2 + i;
    const double *xn = xk + NB;
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      acc = fma(-Ek[j * NB], xn[j], acc);
      w = fmaf(abs_f32_approx(Ek[j * NB]), abs_f32_approx(xn[j]), w);
    }
  }
  if (k == 0) {   // block (1, root) = C_s^T
    const double *Cs = m.C + (size_t)s * nr * NB + i;
    const double *x0 = x + n0;
    for (int j = 0; j < nr; ++j) {
      acc = fma(-Cs[j * NB], x0[j], acc);
      w = fmaf(abs_f32_approx(Cs[j * NB]), abs_f32_approx(x0[j]), w);
    }
  }
  m.rho[off + i] = acc;
  return omega_of(acc, w);
}

// Float-float residual (refinement with ffres = 1). The FP64 entries of K
// and x are split into hi + lo floats (|v - hi - lo| <= 2^-48 |v|). Per
// term, hi*hi is formed exactly (TwoProduct, bm_ff.cuh) and its high part
// summed with TwoSum; the rounding errors of both and the cross terms
// hi*lo + lo*hi go to a low FP32 sum (lo*lo, below 2^-48 |K||x|, is
// dropped). Every 8 terms both sums are added to an FP64 accumulator, so
// the low sum never holds more than 8 terms' worth:
//   |rho_ff - rho|_i <= (8 * 4 * 11 + 3) 2^-48 (|K||x|)_i + O(2^-53)
//                    ~ 1.3e-12 (|K||x|)_i,
// below kFFBeta. With the stopping test omega <= tol - kFFBeta the exact
// omega of an accepted iterate is <= tol.
constexpr double kFFBeta = 4e-12;
// Smallest tolerance refined with float-float residuals (2.5 kFFBeta): the
// stopping test then still accepts omega up to 0.6 tol.
constexpr double kFFMinTol = 1e-11;

template <int NB, int STRIDE>
__device__ __forceinline__ void ff_block(double &acc, float &w, const float *__restrict__ kh,
                                         const float *__restrict__ kl, const float *__restrict__ xh,
                                         const float *__restrict__ xl) {
  constexpr bool V4 = STRIDE == 1 && NB % 4 == 0;
#pragma unroll
  for (int j0 = 0; j0 < NB; j0 += 8) {
    constexpr int CH = 8;
    float a[CH], al[CH], b[CH], bl[CH];
    const int cnt = NB - j0 < CH ? NB - j0 : CH;
    if constexpr (V4) {
#pragma unroll
      for (int g = 0; g < CH / 4; ++g) {
        if (4 * g < cnt) {
          const float4 va = *reinterpret_cast<const float4 *>(kh + j0 + 4 * g);
          const float4 vl = *reinterpret_cast<const float4 *>(kl + j0 + 4 * g);
          const float4 vb = __ldg(reinterpret_cast<const float4 *>(xh + j0 + 4 * g));
          const float4 vc = __ldg(reinterpret_cast<const float4 *>(xl + j0 + 4 * g));
          a[4 * g] = va.x; a[4 * g + 1] = va.y; a[4 * g + 2] = va.z; a[4 * g + 3] = va.w;
          al[4 * g] = vl.x; al[4 * g + 1] = vl.y; al[4 * g + 2] = vl.z; al[4 * g + 3] = vl.w;
          b[4 * g] = vb.x; b[4 * g + 1] = vb.y; b[4 * g + 2] = vb.z; b[4 * g + 3] = vb.w;
          bl[4 * g] = vc.x; bl[4 * g + 1] = vc.y; bl[4 * g + 2] = vc.z; bl[4 * g + 3] = vc.w;
        }
      }
    } else {
#pragma unroll
      for (int t = 0; t < CH; ++t) {
        if (t < cnt) {
          a[t] = kh[(j0 + t) * STRIDE];
          al[t] = kl[(j0 + t) * STRIDE];
          b[t] = __ldg(xh + j0 + t);
          bl[t] = __ldg(xl + j0 + t);
        }
      }
    }
    float sh = 0.0f, c = 0.0f;
#pragma unroll
    for (int t = 0; t < CH; ++t) {
      if (t < cnt) {
        float p, ep, es;
        ff::two_prod(a[t], b[t], p, ep);
        ff::two_sum(sh, p, sh, es);
        c = __fadd_rn(c, __fadd_rn(es, ep));
        c = __fmaf_rn(a[t], bl[t], c);
        c = __fmaf_rn(al[t], b[t], c);
        w = __fmaf_rd(fabsf(a[t]), fabsf(b[t]), w);
      }
    }
    acc += f2d_exact(sh);
    acc += f2d_exact(c);
  }
}

// Row i of block row (s, k) of the residual in float-float; as
// residual_row, but (|K||x|)_i from the hi parts (scaled down by 2^-22 to
// cover their rounding, so omega is never understated).
template <int NB>
__device__ __forceinline__ float residual_row_ff(const MixedState &m, const double *__restrict__ r,
                                                 const double *__restrict__ x, int s, int k, int i) {
  constexpr int NB2 = NB * NB;
  const int N = m.N, nr = m.nr;
  const size_t n0 = (size_t)m.S * N * NB;
  const long br = (long)s * N + k;
  const size_t off = (size_t)br * NB;
  double acc = 0.0;
  float w = 0.0f;
  {
    const size_t kb = (size_t)br * NB2 + (size_t)i * NB;
    ff_block<NB, 1>(acc, w, m.Kdh + kb, m.Kdl + kb, m.xh + off, m.xl + off);
  }
  if (k > 0) {   // block (k, k-1) = E_k: row i
    const size_t eb = ((size_t)s * (N - 1) + (k - 1)) * NB2 + (size_t)i * NB;
    ff_block<NB, 1>(acc, w, m.Keh + eb, m.Kel + eb, m.xh + off - NB, m.xl + off - NB);
  }
  if (k + 1 < N) {   // block (k, k+1) = E_{k+1}^T: column i of E_{k+1}
    const size_t eb = ((size_t)s * (N - 1) + k) * NB2 + i;
    ff_block<NB, NB>(acc, w, m.Keh + eb, m.Kel + eb, m.xh + off + NB, m.xl + off + NB);
  }
  const double ri = r[off + i];
  double rho = ri - acc;
  w = __fadd_rd(__fmul_rd(w, __int_as_float(0x3f7ffffc)), abs_f32_approx(ri));   // 1 - 2^-22
  if (k == 0) {   // block (1, root) = C_s^T, in FP64
    const double *Cs = m.C + (size_t)s * nr * NB + i;
    const double *x0 = x + n0;
    for (int j = 0; j < nr; ++j) {
      rho = fma(-Cs[j * NB], x0[j], rho);
      w = fmaf(abs_f32_approx(Cs[j * NB]), abs_f32_approx(x0[j]), w);
    }
  }
  m.rho[off + i] = rho;
  return omega_of(rho, w);
}

// Folds a lane's omega into the warp and then into the system's wmax.
__device__ __forceinline__ void omega_publish(IRCtl *ctl, float om) {
  unsigned b = __float_as_uint(om);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned v = __shfl_xor_sync(0xffffffffu, b, o);
    b = v > b ? v : b;
  }
  if ((threadIdx.x & 31) == 0 && b) atomicMax(&ctl->wmax, b);
}

// rho = r - K x for the rows of tail s (one CTA per tail) and their omega.
// One thread per row of the tail, so that every lane of an FP64 warp
// instruction does useful work (the FP64 pipe charges whole warps).
template <int NB>
__device__ __forceinline__ void residual_tail(const MixedState &m, const double *__restrict__ r,
                                              const double *__restrict__ x, int s) {
  float om = 0.0f;
  const int rows = m.N * NB;
  for (int e = threadIdx.x; e < rows; e += blockDim.x) {
    const int k = e / NB, i = e - k * NB;
    om = fmaxf(om, residual_row<NB>(m, r, x, s, k, i));
  }
  omega_publish(m.ctl, om);
}

// Root row c of the residual, by one CTA: rho_0c = r_0c - (R x_0)_c -
// sum_i (C_i x_1^i)_c, stored in m.rho; returns omega_c to thread 0. The sum
// is fixed in order whatever the CTA's size (up to 256 threads): 256
// virtual lanes each add the terms e = lane, lane + 256, ... in increasing
// e, and the 256 partial sums are combined by a fixed halving tree.
__device__ __forceinline__ float residual_root_row(const MixedState &m, const double *__restrict__ r,
                                                   const double *__restrict__ x, int NBr, int c) {
  __shared__ double red[256];
  __shared__ float redf[256];
  const int N = m.N, nr = m.nr, S = m.S;
  const size_t n0 = (size_t)S * N * NBr;
  const double *C = m.C, *R = m.R, *x0 = x + n0;
  const long nterm = (long)S * NBr + nr;
  for (int vl = threadIdx.x; vl < 256; vl += blockDim.x) {
    double acc = 0.0;
    float w = 0.0f;
    for (long e = vl; e < nterm; e += 256) {
      double kv, xv;
      if (e < (long)S * NBr) {
        const int s = (int)(e / NBr), j = (int)(e - (long)s * NBr);
        kv = C[((size_t)s * nr + c) * NBr + j];
        xv = x[(size_t)s * N * NBr + j];
      } else {
        const int j = (int)(e - (long)S * NBr);
        kv = j <= c ? R[c * nr + j] : R[j * nr + c];
        xv = x0[j];
      }
      acc = fma(kv, xv, acc);
      w = fmaf(abs_f32_approx(kv), abs_f32_approx(xv), w);
    }
    red[vl] = acc;
    redf[vl] = w;
  }
  for (int h = 128; h > 0; h >>= 1) {
    __syncthreads();
    for (int t = threadIdx.x; t < h; t += blockDim.x) {
      red[t] += red[t + h];
      redf[t] += redf[t + h];
    }
  }
  __syncthreads();
  float om = 0.0f;
  if (threadIdx.x == 0) {
    const double rc = r[n0 + c] - red[0];
    m.rho[n0 + c] = rc;
    om = omega_of(rc, redf[0] + abs_f32_approx(r[n0 + c]));
  }
  __syncthreads();
  return om;
}

// The stopping test of one refinement iteration, by one thread once every
// row's omega is in: converged when omega <= tol; BM_ERR_NOT_CONVERGED after
// max_iter corrections, or earlier when omega fails to halve (stalled or
// diverging refinement), which also stops the remaining launches. Returns
// true when another iteration is to run.
__device__ __forceinline__ bool ir_stop(const MixedState &m, float root_omega, int iter, int max_iter, double tol) {
  IRCtl *ctl = m.ctl;
  const unsigned wb = atomicAdd(&ctl->wmax, 0u);
  const float wf = fmaxf(__uint_as_float(wb), root_omega);
  const double omega = (double)wf;
  ctl->eta = omega;
  ctl->iters = iter;
  m.status->eta = omega;
  m.status->iters = iter;
  if (omega <= tol) {
    ctl->converged = 1;
  } else if (iter >= max_iter || (iter >= 1 && !(omega <= 0.5 * ctl->omega_prev))) {
    if (m.status->code == 0) m.status->code = (int)BM_ERR_NOT_CONVERGED;
    ctl->converged = 1;
  }
  ctl->omega_prev = omega;
  ctl->wmax = 0u;
  ctl->loop = iter + 1;
  return ctl->converged == 0;
}

// Root rows and the stopping test of one system, by its last CTA.
__device__ __forceinline__ void residual_finish(const MixedState &m, const double *__restrict__ r,
                                                const double *__restrict__ x, int NBr, int iter, int max_iter,
                                                double tol) {
  float om = 0.0f;
  for (int c = 0; c < m.nr; ++c) om = fmaxf(om, residual_root_row(m, r, x, NBr, c));
  if (threadIdx.x == 0) ir_stop(m, om, iter, max_iter, tol);
}

}  // namespace mx
}  // namespace bm
