// Double-word ("double-float") arithmetic: a value is hi + lo, two binary32 numbers with
// |lo| <= ulp(hi)/2, about 48 significant bits, computed on the FP32 pipes.  Used where
// pointwise work needs more than FP32 but FP64 issue slots are the bound (one FP64 warp
// instruction per 64 cycles per SM sub-partition on this part, FP32<->FP64 conversions
// included).
//
// Operations follow Joldes, Muller and Popescu, "Tight and rigorous error bounds for basic
// building blocks of double-word arithmetic" (ACM TOMS 2017): the accurate double-word sum
// (TwoSum of the high and of the low parts, two FastTwoSum renormalisations; relative
// error below 3u^2, u = 2^-24) and the FMA-based products, double word x double word
// without the lo x lo term and double word x binary32, with relative errors of a few u^2
// (the CPU checks bound them by 7u^2 and 4u^2).  Every step is an
// explicit round-to-nearest operation, so multiply-add contraction cannot break the
// error-free transformations.  Conversions to and from binary64 move the fields of the
// IEEE 754 encodings with integer operations (one FP64 add per value stored back).
//
// The functions compile for the device and for the host; the host versions (plain IEEE
// binary32 arithmetic, memcpy bit casts) serve the CPU checks of this header against
// exact rational arithmetic.
#pragma once

#include <math.h>
#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define GPSOC_DW __host__ __device__ __forceinline__
#else
#define GPSOC_DW inline
#endif

namespace gpsoc {

struct DF { float hi, lo; };

// round-to-nearest binary32 operations and bit casts
GPSOC_DW float rn_add(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
GPSOC_DW float rn_sub(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}
GPSOC_DW float rn_mul(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
GPSOC_DW float rn_fma(float a, float b, float c) {
#if defined(__CUDA_ARCH__)
  return __fmaf_rn(a, b, c);
#else
  return fmaf(a, b, c);
#endif
}
GPSOC_DW unsigned f_bits(float f) {
#if defined(__CUDA_ARCH__)
  return __float_as_uint(f);
#else
  unsigned u;
  memcpy(&u, &f, 4);
  return u;
#endif
}
GPSOC_DW float f_from(unsigned u) {
#if defined(__CUDA_ARCH__)
  return __uint_as_float(u);
#else
  float f;
  memcpy(&f, &u, 4);
  return f;
#endif
}
GPSOC_DW unsigned d_hi(double x) {
#if defined(__CUDA_ARCH__)
  return (unsigned)__double2hiint(x);
#else
  uint64_t b;
  memcpy(&b, &x, 8);
  return (unsigned)(b >> 32);
#endif
}
GPSOC_DW unsigned d_lo(double x) {
#if defined(__CUDA_ARCH__)
  return (unsigned)__double2loint(x);
#else
  uint64_t b;
  memcpy(&b, &x, 8);
  return (unsigned)(b & 0xffffffffu);
#endif
}
GPSOC_DW double d_from(unsigned hi, unsigned lo) {
#if defined(__CUDA_ARCH__)
  return __hiloint2double((int)hi, (int)lo);
#else
  const uint64_t b = ((uint64_t)hi << 32) | lo;
  double x;
  memcpy(&x, &b, 8);
  return x;
#endif
}

GPSOC_DW DF dw_fast_two_sum(float a, float b) {   // needs exponent(a) >= exponent(b)
  const float s = rn_add(a, b);
  DF r;
  r.hi = s;
  r.lo = rn_sub(b, rn_sub(s, a));
  return r;
}
GPSOC_DW DF dw_two_sum(float a, float b) {
  const float s = rn_add(a, b);
  const float bb = rn_sub(s, a);
  DF r;
  r.hi = s;
  r.lo = rn_add(rn_sub(a, rn_sub(s, bb)), rn_sub(b, bb));
  return r;
}
GPSOC_DW DF dw_add(DF a, DF b) {
  const DF sh = dw_two_sum(a.hi, b.hi);
  const DF sl = dw_two_sum(a.lo, b.lo);
  const DF v = dw_fast_two_sum(sh.hi, rn_add(sh.lo, sl.hi));
  return dw_fast_two_sum(v.hi, rn_add(sl.lo, v.lo));
}
GPSOC_DW DF dw_neg(DF a) {
  DF r;
  r.hi = -a.hi;
  r.lo = -a.lo;
  return r;
}
GPSOC_DW DF dw_sub(DF a, DF b) { return dw_add(a, dw_neg(b)); }
GPSOC_DW DF dw_mul(DF a, DF b) {
  const float ch = rn_mul(a.hi, b.hi);
  const float cl = rn_fma(a.hi, b.hi, -ch);                       // TwoProd: a.hi b.hi = ch + cl
  const float t = rn_fma(a.lo, b.hi, rn_mul(a.hi, b.lo));
  return dw_fast_two_sum(ch, rn_add(cl, t));
}
GPSOC_DW DF dw_mulf(DF a, float b) {
  const float ch = rn_mul(a.hi, b);
  const float cl = rn_fma(a.lo, b, rn_fma(a.hi, b, -ch));
  return dw_fast_two_sum(ch, cl);
}

// binary32 -> binary64, exact for normal values, zero, inf and NaN (FP32 subnormals, below
// 2^-126, become signed zeros)
GPSOC_DW double widen_f(float f) {
  const unsigned u = f_bits(f);
  const unsigned e = u & 0x7f800000u, sign = u & 0x80000000u;
  // exponent field rebiased by 1023 - 127 = 896, mantissa moved to the top of 52 bits
  unsigned hi = sign | (((u & 0x7fffffffu) >> 3) + 0x38000000u);
  unsigned lo = u << 29;
  if (e == 0u) { hi = sign; lo = 0u; }
  if (e == 0x7f800000u) hi |= 0x7ff00000u;   // inf and NaN stay non-finite
  return d_from(hi, lo);
}
// binary64 -> double word: hi = x rounded to 24 significant bits (half-ulp ties up),
// lo = x - hi rounded to FP32, so |lo| <= ulp(hi)/2 and hi + lo = x to 2^-48 relative
// (a double word holds 48 of the 53 bits).  The 29 low bits of x become FP32 values by
// exact subtractions 1.m 2^q - 2^q, which normalise them.  Finite x with |x| < 2^-126
// gives 0 (its low word vanishes below 2^-80); x beyond the FP32 range gives inf, NaN
// stays NaN.
GPSOC_DW DF dw_of(double x) {
  const unsigned H = d_hi(x), L = d_lo(x);
  const unsigned sign = H & 0x80000000u;
  const int E = (int)((H >> 20) & 0x7ffu);                   // biased binary64 exponent
  const unsigned up = (L >> 28) & 1u;                          // first dropped bit: round up
  DF r;
  // the carry of the rounding runs into the exponent field by itself
  r.hi = f_from((sign | ((unsigned)(E - 896) << 23) | ((H & 0xfffffu) << 3) | (L >> 29)) + up);
  // bits 28..6 of L, weight 2^(E-1069) each: (1 + m 2^-23) 2^(E-1046) - 2^(E-1046), less one
  // more 2^(E-1046) (the unit added to hi) when rounded up
  const unsigned t1 = sign | ((unsigned)(E - 919) << 23);
  const float a = rn_sub(f_from(t1 | ((L >> 6) & 0x7fffffu)), f_from(t1 + (up << 23)));
  // bits 5..0 of L, weight 2^(E-1075): (1 + m 2^-6) 2^(E-1069) - 2^(E-1069)
  const unsigned t2 = sign | ((unsigned)(E - 942) << 23);
  const float b = rn_sub(f_from(t2 | ((L & 0x3fu) << 17)), f_from(t2));
  r.lo = (E >= 943) ? rn_add(a, b) : ((E >= 920) ? a : 0.0f);
  if (E < 897) r.hi = f_from(sign);
  if (E > 1150) {
    r.hi = (E == 2047 && ((H & 0xfffffu) | L) != 0u) ? f_from(0x7fc00000u) : f_from(sign | 0x7f800000u);
    r.lo = 0.0f;
  }
  return r;
}
// double word -> binary64, correctly rounded: one FP64 add of the two exact widenings
GPSOC_DW double dw_to_double(DF a) { return widen_f(a.hi) + widen_f(a.lo); }
// hi and lo of an FP64 value by FP64 arithmetic, for state fields the double-word
// kernels read (set once per step by a scalar step)
GPSOC_DW void dw_split(double x, float* hl) {
  hl[0] = (float)x;
  hl[1] = (float)(x - (double)hl[0]);
}

}  // namespace gpsoc
