// Exact FP32 -> FP64 and rounding FP64 -> FP32 conversions on the integer
// pipe (IEEE-754 bit layouts), keeping the FP64 pipe for arithmetic (a
// hardware conversion costs about as much as an FP64 multiply on this part).
// Zero and FP32 denormals map to signed zero; infinities and NaNs keep their
// class.  Also float-float arithmetic on the FP32 pipe.  Shared by the
// (2+1)-d and (3+1)-d kernels.
#pragma once
#include <cuda_runtime.h>

namespace rlbm {

__device__ __forceinline__ double f2d(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned sgn = b & 0x80000000u;
  const unsigned e = (b >> 23) & 0xFFu;
  const unsigned man = b & 0x7FFFFFu;
  unsigned hi = sgn | ((e + 896u) << 20) | (man >> 3);
  unsigned lo = man << 29;
  hi = (e == 0u) ? sgn : ((e == 0xFFu) ? (sgn | 0x7FF00000u | (man >> 3)) : hi);
  lo = (e == 0u) ? 0u : lo;
  return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ float d2f(double d) {
  // round to nearest (ties away from zero) on the magnitude bits: adding half
  // of the discarded 29-bit tail carries into mantissa and exponent as needed
  // (32-bit halves with an explicit carry keep this on the integer pipe)
  const unsigned lo = (unsigned)__double2loint(d);
  const unsigned hw = (unsigned)__double2hiint(d);
  const unsigned sgn = hw & 0x80000000u;
  unsigned hi = hw & 0x7FFFFFFFu;
  const unsigned ed = hi >> 20;
  const unsigned lo2 = lo + (1u << 28);
  hi += (lo2 < lo) ? 1u : 0u;
  const int e = (int)(hi >> 20) - 896;
  const unsigned man = ((hi & 0xFFFFFu) << 3) | (lo2 >> 29);
  unsigned b = sgn | ((unsigned)e << 23) | man;
  const bool is_nan = (ed == 0x7FFu) && (((hw & 0xFFFFFu) | lo) != 0u);
  const unsigned special = is_nan ? 0x7FC00000u : (sgn | 0x7F800000u);
  b = (e <= 0) ? sgn : ((e >= 255 || ed == 0x7FFu) ? special : b);
  return __uint_as_float(b);
}

// Float-float arithmetic: a value is the unevaluated sum hi + lo of two FP32
// numbers (about 48 significant bits), built on error-free transformations
// (Knuth's two-sum, the FMA two-product).  It runs on the FP32 pipe, whose
// rate is 64 times the FP64 rate on this part.  ff_add and ff_sub are the
// "sloppy" sums: their error is a few units of 2^-48 of the larger operand,
// also under cancellation.  Valid while no intermediate over- or underflows.
struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff ff_sum(float a, float b) {       // exact a + b
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ ff ff_fast(float a, float b) {      // exact a + b for |a| >= |b|
  const float s = a + b;
  return {s, b - (s - a)};
}

__device__ __forceinline__ ff ff_prod(float a, float b) {      // exact a * b
  const float p = __fmul_rn(a, b);     // never contracted into an FMA with a later sum
  return {p, fmaf(a, b, -p)};
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const ff s = ff_sum(a.hi, b.hi);
  return ff_fast(s.hi, s.lo + (a.lo + b.lo));
}

__device__ __forceinline__ ff ff_sub(ff a, ff b) {
  const ff s = ff_sum(a.hi, -b.hi);
  return ff_fast(s.hi, s.lo + (a.lo - b.lo));
}

// The products are left unnormalised (|lo| may exceed half an ulp of hi by a
// few units of 2^-24 |lo|); the sums above accept such operands.
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const ff p = ff_prod(a.hi, b.hi);
  return {p.hi, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo))};
}

__device__ __forceinline__ ff ff_mulf(float a, ff b) {
  const ff p = ff_prod(a, b.hi);
  return {p.hi, fmaf(a, b.lo, p.lo)};
}

}  // namespace rlbm
