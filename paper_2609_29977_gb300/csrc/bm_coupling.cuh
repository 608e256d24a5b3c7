// Refined coupling columns of the mixed-precision factor.
//
// The root Schur complement of Alg. 1 steps 3-4, R~ = R - sum_i U_i with
// U_i = C_{i,1} (K_i^{-1})_{11} C_{i,1}^T, is a difference of large terms on
// barrier-scaled systems: ||sum_i U_i|| reaches 10^4 ||R~|| (the generator
// makes R~ = R0 exactly). FP32 tail factors give each U_i only to about
// 1e-5, so the FP32-based R~ can be wrong by O(1). What must be accurate is
// therefore only X_i = K_i^{-1} C_i^T, the nr columns through which tail i
// meets the root (C_i^T is C_{i,1}^T on the rows of stage 1, zero elsewhere;
// Theorem 1 shows that only the x_1 block of the factor couples to the
// root). They are computed with the FP32 tail factor L^ and one step of
// iterative refinement whose residual is exact to about 2^-46:
//   X0 = L^-T L^-1 C_i^T               (FP32, nr right-hand sides),
//   P  = C_i^T - K_i X0                (float-float: Dot2 on split FP64 blocks),
//   X  = X0 + L^-T L^-1 P              (FP32 solve, X0 + d kept as a pair),
//   U_i = sym(C_{i,1} X_{(1)})         (FP64 from the pair X0 + d).
// The solve then uses X_i directly (bm_mixed.cuh): the root right-hand side
// is r_0 - sum_i X_i^T r_i and the tails get L^-T L^-1 r_i - X_i x_0, so the
// FP32 tail solves no longer enter the root step and refinement converges
// at the rate of the FP32 tail factor alone.
//
// Multi right-hand-side tail solves: the same level walk as the solve of
// Alg. 2 (bm_mixed.cuh), with each lane of a team holding one block row for
// RC right-hand sides at a time. Vectors are [S][N][nb][ldc] floats, natural
// stage order, ldc = nr rounded up to RC. The right-hand sides of the
// neighbours' contributions are staged in shared memory per team.
#pragma once

#include "bm_ff.cuh"
#include "bm_mixed.cuh"

namespace bm {
namespace cx {

constexpr int RC = 8;   // right-hand sides per register chunk

struct CxView {
  int S, N, nr, ldc, Lc;
  const float *Ld, *Ll, *Lr, *invd;   // FP32 tail factor
  const double *D, *E, *C;            // FP64 inputs
  float *Xa;   // [S][N][nb][ldc] X0, then the refined X (rounded to FP32)
  float *Yb;   // [S][N][nb][ldc] forward vectors, then the correction d
  float *Zr;   // [S][N][nb][ldc] residual P, then partial gathers in place
  double *U;   // [S][nr][nr]
  const int *on;  // refinement engaged (device word); null: always
};

__device__ __forceinline__ bool engaged(const CxView &v) {
  return v.on == nullptr || *((volatile const int *)v.on) != 0;
}

__device__ __forceinline__ float4 ld4cg(const float *p) { return __ldcg(reinterpret_cast<const float4 *>(p)); }
__device__ __forceinline__ float4 ld4s(const float *p) { return *reinterpret_cast<const float4 *>(p); }

// Team copy of an NB x RC chunk of a vector block (rows of ldc floats, from
// column c0) into shared memory [NB][RC], through L2.
template <int NB, int TS>
__device__ __forceinline__ void stage_chunk(float *__restrict__ dst, const float *src, int ldc, int lane) {
  constexpr int Q = NB * RC / 4;
#pragma unroll
  for (int e = lane; e < Q; e += TS) {
    const int k = e / (RC / 4), g = e - k * (RC / 4);
    *reinterpret_cast<float4 *>(dst + k * RC + 4 * g) = ld4cg(src + (size_t)k * ldc + 4 * g);
  }
}

// z[c] -= sum_k l[k] sY[k][c]
template <int NB>
__device__ __forceinline__ void gather_chunk(float (&z)[RC], const float (&l)[NB], const float *sY) {
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    const float4 a = ld4s(sY + k * RC), b = ld4s(sY + k * RC + 4);
    z[0] = fmaf(-l[k], a.x, z[0]);
    z[1] = fmaf(-l[k], a.y, z[1]);
    z[2] = fmaf(-l[k], a.z, z[2]);
    z[3] = fmaf(-l[k], a.w, z[3]);
    z[4] = fmaf(-l[k], b.x, z[4]);
    z[5] = fmaf(-l[k], b.y, z[5]);
    z[6] = fmaf(-l[k], b.z, z[6]);
    z[7] = fmaf(-l[k], b.w, z[7]);
  }
}

// Row i (l[k] = L[i][k]) or column i (l[k] = L[k][i]) of a block.
template <int NB>
__device__ __forceinline__ void load_col(float (&l)[NB], const float *__restrict__ Lblk, int i) {
#pragma unroll
  for (int k = 0; k < NB; ++k) l[k] = Lblk[k * NB + i];
}

// z := L^{-1} z with the diagonal block distributed by rows (lane i holds
// row i in l[] and 1/L_ii in inv); sx: [NB][RC] team scratch (wide teams).
template <int NB, int TS>
__device__ __forceinline__ void diag_fwd(float (&z)[RC], const float (&l)[NB], float inv, int i, const Team<TS> &tm,
                                         float *sx) {
  if constexpr (TS <= 32) {
    const int base = (threadIdx.x & 31) & ~(TS - 1);
#pragma unroll
    for (int j = 0; j < NB; ++j) {
#pragma unroll
      for (int c = 0; c < RC; ++c) {
        if (i == j) z[c] *= inv;
        const float yj = __shfl_sync(tm.mask, z[c], base + j);
        if (i > j && i < NB) z[c] = fmaf(-l[j], yj, z[c]);
      }
    }
  } else {
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      if (i == j) {
#pragma unroll
        for (int c = 0; c < RC; ++c) {
          z[c] *= inv;
          sx[j * RC + c] = z[c];
        }
      }
      tm.sync();
      if (i > j && i < NB) {
        const float4 a = ld4s(sx + j * RC), b = ld4s(sx + j * RC + 4);
        const float yv[RC] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
        for (int c = 0; c < RC; ++c) z[c] = fmaf(-l[j], yv[c], z[c]);
      }
    }
  }
}

// z := L^{-T} z with lane i holding column i of L (l[k] = L[k][i]).
template <int NB, int TS>
__device__ __forceinline__ void diag_bwd(float (&z)[RC], const float (&l)[NB], float inv, int i, const Team<TS> &tm,
                                         float *sx) {
  if constexpr (TS <= 32) {
    const int base = (threadIdx.x & 31) & ~(TS - 1);
#pragma unroll
    for (int j = NB - 1; j >= 0; --j) {
#pragma unroll
      for (int c = 0; c < RC; ++c) {
        if (i == j) z[c] *= inv;
        const float xj = __shfl_sync(tm.mask, z[c], base + j);
        if (i < j) z[c] = fmaf(-l[j], xj, z[c]);
      }
    }
  } else {
#pragma unroll
    for (int j = NB - 1; j >= 0; --j) {
      if (i == j) {
#pragma unroll
        for (int c = 0; c < RC; ++c) {
          z[c] *= inv;
          sx[j * RC + c] = z[c];
        }
      }
      tm.sync();
      if (i < j) {
        const float4 a = ld4s(sx + j * RC), b = ld4s(sx + j * RC + 4);
        const float xv[RC] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
        for (int c = 0; c < RC; ++c) z[c] = fmaf(-l[j], xv[c], z[c]);
      }
    }
  }
}

template <int NB>
struct XCfg {
  static constexpr int TS = mx::MCfg<NB>::TS;
  // CTAs of four one-warp teams for nb > 16: at up to 128 registers four
  // such CTAs share an SM, so that the 512 tails of the mixed workload run
  // in one wave (eight-team CTAs fit two per SM: 1.7 waves)
  static constexpr int THREADS = TS >= 32 ? 128 : 256;
  static constexpr int MINB = TS >= 32 ? 4 : 2;
  static constexpr int TEAMS = THREADS / TS;
  static constexpr int SCR = 3 * NB * RC;   // per-team scratch floats: two neighbours + diagonal exchange
};

// Forward substitution L^ y = P of one tail for all ldc right-hand sides
// (the levels of Gamma_{N-1} upwards, then x_1). P is read from Zr, where
// positions that are not yet eliminated keep their partial sums; y goes to
// Yb. The CTAs of a cluster (CS of them) split each level's positions.
template <int NB>
__device__ __forceinline__ void fwd_multi(const CxView &v, int s, int crank, int CS, float *scr) {
  constexpr int TS = XCfg<NB>::TS, TEAMS = XCfg<NB>::TEAMS, NB2 = NB * NB;
  const Team<TS> tm;
  const int N = v.N, Lc = v.Lc, ldc = v.ldc;
  const size_t sb = (size_t)s * N;
  const int i = tm.lane, ir = i < NB ? i : 0;
  float *s0 = scr + tm.id * XCfg<NB>::SCR, *s1 = s0 + NB * RC, *sx = s1 + NB * RC;
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
      int pl = 0, pr = 0;
      if (lvl >= 1) {
        const int h = 1 << (lvl - 1);
        if (q < N) {
          pl = q - h;
          if (q + h <= N - 1) pr = q + h;
        } else {
          const int mm = ((N - 1) >> (lvl - 1)) << (lvl - 1);
          if (ctz32(mm) == lvl - 1) pl = mm;
        }
      }
      const float inv = elim ? v.invd[(sb + (N - q)) * NB + ir] : 0.0f;
      const size_t row = ((sb + (N - q)) * NB + ir) * ldc;
      for (int c0 = 0; c0 < ldc; c0 += RC) {
        // one register row at a time (the first one loaded ahead of the
        // staging barrier), so that two CTAs fit on an SM
        float l[NB];
        if (pl) mx::load_row<NB>(l, v.Lr + (sb + (N - pl)) * NB2 + ir * NB);
        if (pl) stage_chunk<NB, TS>(s0, v.Yb + (sb + (N - pl)) * NB * ldc + c0, ldc, i);
        if (pr) stage_chunk<NB, TS>(s1, v.Yb + (sb + (N - pr)) * NB * ldc + c0, ldc, i);
        float z[RC];
        {
          const float4 a = ld4cg(v.Zr + row + c0), b = ld4cg(v.Zr + row + c0 + 4);
          z[0] = a.x; z[1] = a.y; z[2] = a.z; z[3] = a.w; z[4] = b.x; z[5] = b.y; z[6] = b.z; z[7] = b.w;
        }
        tm.sync();
        if (pl) gather_chunk<NB>(z, l, s0);
        if (pr) {
          mx::load_row<NB>(l, v.Ll + (sb + (N - pr)) * NB2 + ir * NB);
          gather_chunk<NB>(z, l, s1);
        }
        float *dst = v.Zr;
        if (elim) {
          mx::load_row<NB>(l, v.Ld + (sb + (N - q)) * NB2 + ir * NB);
          diag_fwd<NB, TS>(z, l, inv, i, tm, sx);
          dst = v.Yb;
        }
        if (i < NB) {
          *reinterpret_cast<float4 *>(dst + row + c0) = make_float4(z[0], z[1], z[2], z[3]);
          *reinterpret_cast<float4 *>(dst + row + c0 + 4) = make_float4(z[4], z[5], z[6], z[7]);
        }
        tm.sync();
      }
    }
    if (CS > 1)
      mx::cluster_sync();
    else
      __syncthreads();
  }
}

// Backward substitution L^T x = y of one tail for all ldc right-hand sides,
// from x_1 down the levels.
//  * pass 0 (X0): y is zero except on x_1, where y_1 = L_{i,1}^{-1} C_{i,1}^T
//    (the forward substitution of C_i^T reduces to that block, x_1 being
//    ordered last); the solution X0 goes to Xa.
//  * pass 1 (correction): y is read from Yb and the correction d
//    overwrites it; Xa += d (FP32) and, on x_1, U_i = sym(C_{i,1} (X0 + d))
//    in FP64 from the unrounded pair.
template <int NB>
__device__ __forceinline__ void bwd_multi(const CxView &v, int s, int crank, int CS, int pass, float *scr) {
  constexpr int TS = XCfg<NB>::TS, TEAMS = XCfg<NB>::TEAMS, NB2 = NB * NB;
  const Team<TS> tm;
  const int N = v.N, Lc = v.Lc, ldc = v.ldc, nr = v.nr;
  const size_t sb = (size_t)s * N;
  const int i = tm.lane, ir = i < NB ? i : 0;
  float *s0 = scr + tm.id * XCfg<NB>::SCR, *s1 = s0 + NB * RC, *sx = s1 + NB * RC;
  float *out = pass == 0 ? v.Xa : v.Yb;
  for (int lvl = Lc; lvl >= 0; --lvl) {
    const bool first = lvl == Lc;
    const int ntask = first ? 1 : (((N - 1) >> lvl) + 1) / 2;
    for (int t = crank * TEAMS + tm.id; t < ntask; t += CS * TEAMS) {
      const int q = first ? N : (2 * t + 1) << lvl;
      int a = 0, b = 0;
      if (!first) {
        const int h = 1 << lvl;
        b = (q + h <= N - 1) ? q + h : N;
        if (q > h) a = q - h;
      }
      const float inv = v.invd[(sb + (N - q)) * NB + ir];
      const size_t row = ((sb + (N - q)) * NB + ir) * ldc;
      for (int c0 = 0; c0 < ldc; c0 += RC) {
        // one register column at a time (the first one loaded ahead of the
        // staging barrier), so that two CTAs fit on an SM
        float l[NB];
        if (b) load_col<NB>(l, v.Lr + (sb + (N - q)) * NB2, ir);
        if (b) stage_chunk<NB, TS>(s0, out + (sb + (N - b)) * NB * ldc + c0, ldc, i);
        if (a) stage_chunk<NB, TS>(s1, out + (sb + (N - a)) * NB * ldc + c0, ldc, i);
        float z[RC];
        if (pass == 1) {
          const float4 u = ld4cg(v.Yb + row + c0), w = ld4cg(v.Yb + row + c0 + 4);
          z[0] = u.x; z[1] = u.y; z[2] = u.z; z[3] = u.w; z[4] = w.x; z[5] = w.y; z[6] = w.z; z[7] = w.w;
        } else {
#pragma unroll
          for (int c = 0; c < RC; ++c) z[c] = 0.0f;
        }
        if (first && pass == 0) {
          // y_1 = L_{i,1}^{-1} C_{i,1}^T: row i of the diagonal block
          float lrow[NB];
          mx::load_row<NB>(lrow, v.Ld + (sb + (N - q)) * NB2 + ir * NB);
#pragma unroll
          for (int c = 0; c < RC; ++c)
            z[c] = (i < NB && c0 + c < nr) ? __double2float_rn(v.C[((size_t)s * nr + c0 + c) * NB + i]) : 0.0f;
          diag_fwd<NB, TS>(z, lrow, inv, i, tm, sx);
        }
        tm.sync();
        if (b) gather_chunk<NB>(z, l, s0);
        if (a) {
          load_col<NB>(l, v.Ll + (sb + (N - q)) * NB2, ir);
          gather_chunk<NB>(z, l, s1);
        }
        load_col<NB>(l, v.Ld + (sb + (N - q)) * NB2, ir);
        diag_bwd<NB, TS>(z, l, inv, i, tm, sx);
        float x0[RC];
        if (pass == 1) {
          const float4 u = ld4cg(v.Xa + row + c0), w = ld4cg(v.Xa + row + c0 + 4);
          x0[0] = u.x; x0[1] = u.y; x0[2] = u.z; x0[3] = u.w; x0[4] = w.x; x0[5] = w.y; x0[6] = w.z; x0[7] = w.w;
        }
        if (i < NB) {
          *reinterpret_cast<float4 *>(out + row + c0) = make_float4(z[0], z[1], z[2], z[3]);
          *reinterpret_cast<float4 *>(out + row + c0 + 4) = make_float4(z[4], z[5], z[6], z[7]);
          if (pass == 1) {
            *reinterpret_cast<float4 *>(v.Xa + row + c0) =
                make_float4(x0[0] + z[0], x0[1] + z[1], x0[2] + z[2], x0[3] + z[3]);
            *reinterpret_cast<float4 *>(v.Xa + row + c0 + 4) =
                make_float4(x0[4] + z[4], x0[5] + z[5], x0[6] + z[6], x0[7] + z[7]);
          }
        }
        if (first && pass == 1) {
          // U_i[a][c0 + c] = sum_k C[a][k] (X0 + d)[k][c0 + c] in FP64
          tm.sync();
          double *sX = reinterpret_cast<double *>(s0);   // NB x RC doubles fit in s0..s1
          if (i < NB) {
#pragma unroll
            for (int c = 0; c < RC; ++c) sX[i * RC + c] = f2d_exact(x0[c]) + f2d_exact(z[c]);
          }
          tm.sync();
          double *Us = v.U + (size_t)s * nr * nr;
          for (int e = i; e < nr * RC; e += TS) {
            const int ar = e / RC, c = e - ar * RC;
            if (c0 + c >= nr) continue;
            const double *Ca = v.C + ((size_t)s * nr + ar) * NB;
            double acc = 0.0;
#pragma unroll
            for (int k = 0; k < NB; ++k) acc = fma(Ca[k], sX[k * RC + c], acc);
            Us[ar * nr + c0 + c] = acc;
          }
        }
        tm.sync();
      }
      if (first && pass == 1) {
        // U_i := (U_i + U_i^T) / 2 (the exact U_i is symmetric)
        double *Us = v.U + (size_t)s * nr * nr;
        for (int e = i; e < nr * nr; e += TS) {
          const int ar = e / nr, c = e - ar * nr;
          if (c >= ar) continue;
          const double u = 0.5 * (Us[ar * nr + c] + Us[c * nr + ar]);
          Us[ar * nr + c] = u;
          Us[c * nr + ar] = u;
        }
        tm.sync();
      }
    }
    if (CS > 1)
      mx::cluster_sync();
    else
      __syncthreads();
  }
}

// P = C_i^T - K_i X0 for one row (tail s, natural stage k + 1, block row i)
// and all ldc right-hand sides, exact to about 2^-46 relative to
// |C^T| + |K| |X0|: every FP64 entry is split into hi + lo floats and the
// products with the (exactly FP32) X0 are summed by Dot2.
template <int NB>
__device__ __forceinline__ void residual_row_multi(const CxView &v, int s, int k, int i) {
  constexpr int NB2 = NB * NB;
  const int N = v.N, nr = v.nr, ldc = v.ldc;
  const size_t br = (size_t)s * N + k;
  const double *Dk = v.D + br * NB2;
  const float *xk = v.Xa + br * NB * ldc;
  for (int c0 = 0; c0 < ldc; c0 += RC) {
    float sh[RC], sl[RC];
#pragma unroll
    for (int c = 0; c < RC; ++c) {
      sh[c] = 0.0f;
      sl[c] = 0.0f;
      if (k == 0 && c0 + c < nr) ff::split_d(v.C[((size_t)s * nr + c0 + c) * NB + i], sh[c], sl[c]);
    }
    auto block = [&](auto kij_of, const float *xb) {
#pragma unroll 4
      for (int j = 0; j < NB; ++j) {
        float kh, kl;
        ff::split_d(kij_of(j), kh, kl);
        const float4 a = *reinterpret_cast<const float4 *>(xb + (size_t)j * ldc + c0);
        const float4 b = *reinterpret_cast<const float4 *>(xb + (size_t)j * ldc + c0 + 4);
        const float xv[RC] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
        for (int c = 0; c < RC; ++c) ff::dot2_step_split(sh[c], sl[c], -kh, -kl, xv[c]);
      }
    };
    block([&](int j) { return j <= i ? Dk[i * NB + j] : Dk[j * NB + i]; }, xk);
    if (k > 0) {   // block (k, k-1) = E_k
      const double *Ek = v.E + ((size_t)s * (N - 1) + (k - 1)) * NB2 + i * NB;
      block([&](int j) { return Ek[j]; }, xk - NB * ldc);
    }
    if (k + 1 < N) {   // block (k, k+1) = E_{k+1}^T
      const double *Ek = v.E + ((size_t)s * (N - 1) + k) * NB2 + i;
      block([&](int j) { return Ek[j * NB]; }, xk + NB * ldc);
    }
    float *o = v.Zr + (br * NB + i) * ldc + c0;
    float r[RC];
#pragma unroll
    for (int c = 0; c < RC; ++c) r[c] = __fadd_rn(sh[c], sl[c]);
    *reinterpret_cast<float4 *>(o) = make_float4(r[0], r[1], r[2], r[3]);
    *reinterpret_cast<float4 *>(o + 4) = make_float4(r[4], r[5], r[6], r[7]);
  }
}

}  // namespace cx
}  // namespace bm
