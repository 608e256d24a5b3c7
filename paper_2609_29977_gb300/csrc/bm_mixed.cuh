// Mixed-precision solve state and the device bodies shared by the single
// system kernels (bm_mixed.cu) and the batched kernels (bm_batch.cu).
#pragma once

#include "bm_tail_factor.cuh"

namespace bm {

struct IRCtl {
  int converged;                  // set by the residual kernel once eta <= tol
  int iters;                      // corrections applied in the last solve
  unsigned long long rmax, xmax;  // |rho|_inf, |x|_inf of the running iteration (bit patterns)
  unsigned long long kmax, bmax;  // ||K||_inf (computed once per factor), ||r||_inf (once per solve)
  int knorm_valid;
  int pad;
  double eta;
};

struct MixedState {
  int S, N, nb, nr, Lc;
  float *Ld, *Ll, *Lr, *Dt, *W, *invd;   // FP32 tail factor and level workspace
  double *F, *U, *LR, *Rt;               // FP64 root parts
  float *y, *zt;                         // [S][N][nb] solve vectors (y is overwritten by the correction)
  double *tb;                            // [S][nr]
  double *d0;                            // [nr] root correction
  double *rho;                           // [n] residual
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
      float z = 0.0f;
      if (i < NB) {
        z = (lvl <= 1) ? d2f_rn(rhs[zoff + i]) : __ldcg(m.zt + zoff + i);
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
          if (pl) {
            const float *L = m.Lr + (sb + (N - pl)) * NB2 + i * NB;
            const float *y = m.y + (sb + (N - pl)) * NB;
#pragma unroll
            for (int k = 0; k < NB; ++k) z = fmaf(-L[k], __ldcg(y + k), z);
          }
          if (pr) {
            const float *L = m.Ll + (sb + (N - pr)) * NB2 + i * NB;
            const float *y = m.y + (sb + (N - pr)) * NB;
#pragma unroll
            for (int k = 0; k < NB; ++k) z = fmaf(-L[k], __ldcg(y + k), z);
          }
        }
      }
      if (!elim) {
        if (i < NB) m.zt[zoff + i] = z;
        continue;
      }
      float Lrow[NB];
      const float *Ld = m.Ld + (sb + (N - q)) * NB2 + (i < NB ? i : 0) * NB;
#pragma unroll
      for (int k = 0; k < NB; ++k) Lrow[k] = Ld[k];
      const float inv = i < NB ? m.invd[zoff + i] : 0.0f;
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
      if (lastlvl) {
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

// Root step of Alg. 2 for one system, by one CTA once every tail's
// t_i = F_{i,1} y_1 is in tb: r~_0 = rhs_0 - sum_i t_i (fixed order),
// d_0 = L_R^{-T} L_R^{-1} r~_0 (FP64), x_0 += d_0.
template <int NB>
__device__ __forceinline__ void root_step(const MixedState &m, const double *__restrict__ rhs, double *x, int iter,
                                          double *sR) {
  const int N = m.N, nr = m.nr, S = m.S;
  const size_t n0 = (size_t)S * N * NB;
  double *sL = sR, *sz = sR + nr * nr, *sInv = sz + nr;
  for (int e = threadIdx.x; e < nr * nr; e += blockDim.x) sL[e] = __ldcg(m.LR + e);
  // r~_0 = rhs_0 - sum_i t_i, fixed summation order per component
  for (int c = threadIdx.x; c < nr; c += blockDim.x) {
    double acc = rhs[n0 + c];
    for (int t = 0; t < S; ++t) acc -= __ldcg(m.tb + (size_t)t * nr + c);
    sz[c] = acc;
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
  (void)sInv;
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
  for (int lvl = Lc; lvl >= 0; --lvl) {
    const bool first = lvl == Lc;
    const int ntask = first ? 1 : (((N - 1) >> lvl) + 1) / 2;
    for (int t = crank * TEAMS + tm.id; t < ntask; t += CS * TEAMS) {
      const int q = first ? N : (2 * t + 1) << lvl;
      const size_t zoff = (sb + (N - q)) * NB;
      float z = 0.0f;
      if (i < NB) {
        if (first) {
          double zd = f2d_exact(m.y[zoff + i]);
          const double *Fs = m.F + (size_t)s * nr * NB;
          for (int c = 0; c < nr; ++c) zd = fma(-Fs[c * NB + i], __ldcg(m.d0 + c), zd);
          z = d2f_rn(zd);
        } else {
          z = m.y[zoff + i];
          const int h = 1 << lvl;
          const int a = q - h, b = (q + h <= N - 1) ? q + h : N;
          const float *Lb = m.Lr + (sb + (N - q)) * NB2 + i;
          const float *db = m.y + (sb + (N - b)) * NB;
#pragma unroll
          for (int k = 0; k < NB; ++k) z = fmaf(-Lb[k * NB], __ldcg(db + k), z);
          if (q > h) {
            const float *La = m.Ll + (sb + (N - q)) * NB2 + i;
            const float *da = m.y + (sb + (N - a)) * NB;
#pragma unroll
            for (int k = 0; k < NB; ++k) z = fmaf(-La[k * NB], __ldcg(da + k), z);
          }
        }
      }
      float Lcol[NB];
      const float *Ld = m.Ld + (sb + (N - q)) * NB2 + (i < NB ? i : 0);
#pragma unroll
      for (int k = 0; k < NB; ++k) Lcol[k] = Ld[k * NB];
      const float inv = i < NB ? m.invd[zoff + i] : 0.0f;
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
        const double dz = f2d_exact(z);
        x[zoff + i] = iter == 0 ? dz : x[zoff + i] + dz;
      }
      tm.sync();
    }
    if (CS > 1)
      cluster_sync();
    else
      __syncthreads();
  }
}



// rho = r - K x for the rows of tail s (FP64) with the norms of the stopping
// test accumulated into the system's control block (one CTA per tail).
template <int NB>
__device__ __forceinline__ void residual_tail(const MixedState &m, const double *__restrict__ r,
                                              const double *__restrict__ x, int s, int iter) {
  constexpr int TS = MCfg<NB>::TS, TEAMS = MCfg<NB>::TEAMS, NB2 = NB * NB;
  const Team<TS> tm;
  const int N = m.N, nr = m.nr, S = m.S;
  const size_t n0 = (size_t)S * N * NB;
  const bool knorm = !m.ctl->knorm_valid;
  const double *D = m.D, *E = m.E, *C = m.C;
  const double *x0 = x + n0;
  unsigned long long rmax = 0, xmax = 0, bmax = 0;
  float kmax = 0.0f;
  const int i = tm.lane;
  for (int k = tm.id; k < N; k += TEAMS) {
    if (i >= NB) continue;
    const long br = (long)s * N + k;
    const size_t off = (size_t)br * NB;
    const double *Dk = D + (size_t)br * NB2;
    const double *xk = x + off;
    double acc = r[off + i];
    float ks = 0.0f;
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      const double kij = j <= i ? Dk[i * NB + j] : Dk[j * NB + i];
      acc = fma(-kij, xk[j], acc);
      if (knorm) ks += abs_f32_approx(kij);
    }
    if (k > 0) {
      const double *Ek = E + ((size_t)s * (N - 1) + (k - 1)) * NB2 + i * NB;
      const double *xp = xk - NB;
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        acc = fma(-Ek[j], xp[j], acc);
        if (knorm) ks += abs_f32_approx(Ek[j]);
      }
    }
    if (k + 1 < N) {
      const double *Ek = E + ((size_t)s * (N - 1) + k) * NB2 + i;
      const double *xn = xk + NB;
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        acc = fma(-Ek[j * NB], xn[j], acc);
        if (knorm) ks += abs_f32_approx(Ek[j * NB]);
      }
    }
    if (k == 0) {
      const double *Cs = C + (size_t)s * nr * NB + i;
      for (int j = 0; j < nr; ++j) {
        acc = fma(-Cs[j * NB], x0[j], acc);
        if (knorm) ks += abs_f32_approx(Cs[j * NB]);
      }
    }
    m.rho[off + i] = acc;
    const unsigned long long ra = abs_bits(acc), xa = abs_bits(xk[i]);
    rmax = ra > rmax ? ra : rmax;
    xmax = xa > xmax ? xa : xmax;
    if (iter == 0) {
      const unsigned long long ba = abs_bits(r[off + i]);
      bmax = ba > bmax ? ba : bmax;
    }
    kmax = ks > kmax ? ks : kmax;
  }
  rmax = warp_max_u64(rmax);
  xmax = warp_max_u64(xmax);
  bmax = warp_max_u64(bmax);
  unsigned kb = __float_as_uint(kmax);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned w = __shfl_xor_sync(0xffffffffu, kb, o);
    kb = w > kb ? w : kb;
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&m.ctl->rmax, rmax);
    atomicMax(&m.ctl->xmax, xmax);
    if (iter == 0) atomicMax(&m.ctl->bmax, bmax);
    if (knorm) atomicMax(&m.ctl->kmax, (unsigned long long)kb);
  }
}

// Root rows of the residual and the stopping test, by the last CTA of a
// system once all its tail rows are in: rho_0 = r_0 - R x_0 - sum C_i x_1^i,
// eta = ||rho||_inf / (||K||_inf ||x||_inf + ||r||_inf); sets converged.
__device__ __forceinline__ void residual_finish(const MixedState &m, const double *__restrict__ r,
                                                const double *__restrict__ x, int NBr, int iter, int max_iter,
                                                double tol) {
  __shared__ double red[256];
  __shared__ float redf[256];
  const int N = m.N, nr = m.nr, S = m.S;
  const size_t n0 = (size_t)S * N * NBr;
  const bool knorm = !m.ctl->knorm_valid;
  const double *C = m.C, *R = m.R, *x0 = x + n0;
  unsigned long long rmax = 0, xmax = 0, bmax = 0;
  float kmax = 0.0f;
  for (int c = 0; c < nr; ++c) {
    double acc = 0.0;
    float ks = 0.0f;
    for (long e = threadIdx.x; e < (long)S * NBr + nr; e += blockDim.x) {
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
      if (knorm) ks += abs_f32_approx(kv);
    }
    red[threadIdx.x] = acc;
    redf[threadIdx.x] = ks;
    for (int w = blockDim.x >> 1; w > 0; w >>= 1) {
      __syncthreads();
      if ((int)threadIdx.x < w) {
        red[threadIdx.x] += red[threadIdx.x + w];
        redf[threadIdx.x] += redf[threadIdx.x + w];
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const double rc = r[n0 + c] - red[0];
      m.rho[n0 + c] = rc;
      const unsigned long long ra = abs_bits(rc), xa = abs_bits(x0[c]);
      rmax = ra > rmax ? ra : rmax;
      xmax = xa > xmax ? xa : xmax;
      if (iter == 0) {
        const unsigned long long ba = abs_bits(r[n0 + c]);
        bmax = ba > bmax ? ba : bmax;
      }
      kmax = redf[0] > kmax ? redf[0] : kmax;
    }
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  IRCtl *ctl = m.ctl;
  unsigned long long rb = atomicAdd(&ctl->rmax, 0ull), xb = atomicAdd(&ctl->xmax, 0ull);
  unsigned long long bb = atomicAdd(&ctl->bmax, 0ull), kb = atomicAdd(&ctl->kmax, 0ull);
  rb = rb > rmax ? rb : rmax;
  xb = xb > xmax ? xb : xmax;
  if (iter == 0) bb = bb > bmax ? bb : bmax;
  if (knorm) {
    const unsigned kf = __float_as_uint(kmax);
    kb = kb > kf ? kb : kf;
    ctl->kmax = kb;
  }
  ctl->bmax = bb;
  const double rn = __longlong_as_double((long long)rb), xn = __longlong_as_double((long long)xb);
  const double bn = __longlong_as_double((long long)bb), kn = (double)__uint_as_float((unsigned)kb);
  const double eta = rn / (kn * xn + bn);
  ctl->eta = eta;
  ctl->iters = iter;
  ctl->knorm_valid = 1;
  m.status->eta = eta;
  m.status->iters = iter;
  if (eta <= tol)
    ctl->converged = 1;
  else if (iter >= max_iter && m.status->code == 0)
    m.status->code = (int)BM_ERR_NOT_CONVERGED;
  ctl->rmax = 0ull;
  ctl->xmax = 0ull;
}

}  // namespace mx
}  // namespace bm
