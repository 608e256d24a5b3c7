// Float-float (double-word) arithmetic on the FP32 pipe.
//
// GB300 retires one FP64 warp instruction per 64 cycles on each SM
// sub-partition, against one FP32 instruction per cycle, so sums that need
// more than FP32 accuracy are cheaper as unevaluated pairs hi + lo of
// floats than as doubles:
//  * two_sum: Knuth's TwoSum (TAOCP vol. 2, Sec. 4.2.2): s + e = a + b
//    exactly, with s = fl(a + b), in six additions and no branch;
//  * two_prod: the FMA form of Dekker's TwoProduct: p + e = a * b exactly,
//    with p = fl(a * b) and e = fma(a, b, -p);
//  * dot2_step: one step of Dot2 (Ogita, Rump and Oishi, "Accurate sum and
//    dot product", SIAM J. Sci. Comput. 26(6), 2005): the sum is carried as
//    s + c, products enter through two_prod and s is updated by two_sum; the
//    result is as accurate as if computed in twice the working precision
//    and then rounded;
//  * split_d: a double as hi + lo floats (hi = the FP32 rounding, lo the
//    FP32 rounding of d - hi), so |d - hi - lo| <= 2^-48 |d| in the FP32
//    normal range. hi is the hardware conversion (one FP64-pipe
//    instruction, branch-free, so that the loads of a loop of splits are
//    not ordered by a branch); lo comes from the bits with integer
//    instructions.
// Every operation is written with the _rn intrinsics so that the compiler
// neither contracts a product into a later addition nor reorders the sums.
#pragma once

#include "bm_team.cuh"

namespace bm {
namespace ff {

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  const float t = __fadd_rn(a, b);
  const float bp = __fsub_rn(t, a);
  const float ap = __fsub_rn(t, bp);
  e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
  s = t;
}

__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
  const float t = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -t);
  p = t;
}

// (s, c) += a * b.
__device__ __forceinline__ void dot2_step(float &s, float &c, float a, float b) {
  float p, ep, es;
  two_prod(a, b, p, ep);
  two_sum(s, p, s, es);
  c = __fadd_rn(c, __fadd_rn(es, ep));
}

// (s, c) += (ah + al) * b, with al * b carried only in the low part (its
// rounding error is 2^-24 of a term already 2^-24 below the product).
__device__ __forceinline__ void dot2_step_split(float &s, float &c, float ah, float al, float b) {
  float p, ep, es;
  two_prod(ah, b, p, ep);
  two_sum(s, p, s, es);
  c = __fadd_rn(c, __fadd_rn(es, __fmaf_rn(al, b, ep)));
}

// d = hi + lo (+ at most 2^-48 |d|). The hardware rounding for hi, integer
// instructions and one int-to-float conversion for lo; outside the FP32
// normal range lo is 0.
__device__ __forceinline__ void split_d(double d, float &hi, float &lo) {
  hi = __double2float_rn(d);
  const unsigned whi = (unsigned)__double2hiint(d), wlo = (unsigned)__double2loint(d);
  const unsigned e = (whi >> 20) & 0x7ffu;
  lo = 0.0f;
  if (e - 897u < 253u) {
    // d2f_rn kept the top 24 significand bits and rounded on the low 29:
    // the remainder d - hi is rem or rem - 2^29 units of 2^(e - 1075)
    const unsigned rem = wlo & 0x1fffffffu;
    const unsigned kept = ((whi & 0x000fffffu) << 3) | (wlo >> 29);
    const bool up = (rem > 0x10000000u) || (rem == 0x10000000u && (kept & 1u));
    const int r = up ? (int)rem - (int)0x20000000 : (int)rem;
    if (r != 0) {
      const unsigned fb = __float_as_uint(__int2float_rn(r));
      const int fe = (int)((fb >> 23) & 0xffu) + (int)e - 1075;
      if (fe > 0) lo = __uint_as_float(((fb & 0x807fffffu) | ((unsigned)fe << 23)) ^ (whi & 0x80000000u));
    }
  }
}

// The float-float residual's range: nonzero magnitudes in [2^-50, 2^50),
// so that every product of hi and lo parts it forms is a normal float.
__device__ __forceinline__ bool out_of_range(double d) {
  const unsigned hi = (unsigned)__double2hiint(d) & 0x7fffffffu, lo = (unsigned)__double2loint(d);
  const unsigned e = hi >> 20;
  return (hi | lo) != 0u && (e < 1023u - 50u || e >= 1023u + 50u);
}

// hi + lo as a double (exact).
__device__ __forceinline__ double to_double(float hi, float lo) { return f2d_exact(hi) + f2d_exact(lo); }

}  // namespace ff
}  // namespace bm
