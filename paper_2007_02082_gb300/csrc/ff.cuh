// Double-FP32 ("float-float") arithmetic for the FP64-accurate stencil sums of
// the mixed path's outer loops and right-hand sides.
//
// GB300 issues FP32 and 32-bit integer instructions at dozens of times its FP64
// rate, so a stencil sum carried as a pair of FP32 numbers (hi + lo, about 48
// significant bits) costs a fraction of the same sum in FP64.  The building
// blocks are the classic error-free transformations:
//   two-sum (Knuth):         a + b = s + e exactly, s = fl(a + b);
//   two-product (with FMA):  a * b = p + e exactly, p = fl(a * b), e = fma(a, b, -p).
// Every step that must round on its own is written with the _rn intrinsics, so
// the compiler cannot contract a product into a following sum.  Conversions
// between FP64 and FP32 pairs use integer operations on the IEEE-754 bits (the
// conversion instructions share the slow FP64 path).
#pragma once

#include <cstdint>

namespace ibg {

struct ff {
  float h, l;
};

__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

// x as hi + lo: hi = x with its mantissa cut to 24 bits (exact), lo = the
// remaining 29 bits rounded to FP32, so hi + lo is within 2^-48 |x| of x for
// |x| >= 2^-100 (below, lo loses bits to the FP32 subnormal range: within
// 2^-149 absolute).  |x| < 2^-126 reads as 0 (an absolute error below
// 1.2e-38); |x| >= 2^128, infinities and NaN go through the conversion
// instruction.
__device__ __forceinline__ ff dsplit(double x) {
  const unsigned uh = unsigned(__double2hiint(x)), ul = unsigned(__double2loint(x));
  const int e = int((uh >> 20) & 0x7FFu);
  const unsigned sign = uh & 0x80000000u;
  if (e <= 896) return {0.f, 0.f};
  if (e >= 1151) return {__double2float_rn(x), 0.f};
  const float h = __uint_as_float(sign | (unsigned(e - 896) << 23) | ((uh & 0xFFFFFu) << 3) | (ul >> 29));
  // the low 29 mantissa bits r = r1 * 64 + r0, each part < 2^23 made exact by
  // the 2^23 constant, then scaled by 2^(e - 1075) (in two steps where that
  // power of two is below the normal FP32 range)
  const unsigned r = ul & 0x1FFFFFFFu;
  const float r1 = __fsub_rn(__uint_as_float(0x4B000000u | (r >> 6)), 8388608.f);
  const float r0 = __fsub_rn(__uint_as_float(0x4B000000u | (r & 63u)), 8388608.f);
  const float rr = fmaf(r1, 64.f, r0);
  float l = e > 948 ? __fmul_rn(rr, __uint_as_float(unsigned(e - 948) << 23))
                    : __fmul_rn(__fmul_rn(rr, __uint_as_float(unsigned(e - 884) << 23)), 5.421010862427522e-20f);
  l = __uint_as_float(__float_as_uint(l) | sign);
  return {h, l};
}

// f exactly as FP64 (normal FP32 numbers and zeros by their bits).
__device__ __forceinline__ double f2d(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned E = (u >> 23) & 0xFFu;
  if ((u << 1) == 0u) return __hiloint2double(int(u), 0);
  if (E == 0u || E == 255u) return double(f);
  return __hiloint2double(int((u & 0x80000000u) | ((E + 896u) << 20) | ((u & 0x7FFFFFu) >> 3)), int(u << 29));
}

// x * 2^s, exact, by the exponent field where the result stays a normal
// number (zeros pass through); otherwise the library's ldexp.
__device__ __forceinline__ double scale2(double x, int s) {
  const int hw = __double2hiint(x), lw = __double2loint(x);
  const int e = (hw >> 20) & 0x7FF;
  if (e == 0 && ((hw & 0x7FFFFFFF) | lw) == 0) return x;
  if (e > 0 && e < 2047 && e + s > 0 && e + s < 2047) return __hiloint2double(hw + (s << 20), lw);
  return ldexp(x, s);
}

// x rounded to FP32 (nearest) without the conversion instruction, for
// 2^-126 <= |x| < 2^128 (smaller values read as zero)
__device__ __forceinline__ float d2f(double x) {
  const ff p = dsplit(x);
  return __fadd_rn(p.h, p.l);
}

// hi + lo in FP64 (one FP64 addition)
__device__ __forceinline__ double ff2d(ff a) { return f2d(a.h) + f2d(a.l); }

// A small integer (|w| < 2^22) as FP32, exact, without the conversion instruction.
__device__ __forceinline__ float wf(int w) { return __fsub_rn(__int_as_float(0x4B400000 + w), 12582912.f); }

// a += w x for an integer-valued w (|w| < 2^12): the product's rounding error
// (two-product) and the sum's (two-sum) are carried in lo.
__device__ __forceinline__ void ff_madd_int(ff& a, float w, ff x) {
  const float p = __fmul_rn(w, x.h);
  const float pe = fmaf(w, x.h, -p);
  const ff s = two_sum(a.h, p);
  a.h = s.h;
  a.l = __fadd_rn(a.l, __fadd_rn(s.l, fmaf(w, x.l, pe)));
}

// a += c x, c and x pairs (the lo * lo term, below 2^-48 of the product, is dropped)
__device__ __forceinline__ void ff_madd(ff& a, ff c, ff x) {
  const float p = __fmul_rn(c.h, x.h);
  const float pe = fmaf(c.h, x.h, -p);
  const ff s = two_sum(a.h, p);
  a.h = s.h;
  a.l = __fadd_rn(a.l, __fadd_rn(s.l, fmaf(c.h, x.l, fmaf(c.l, x.h, pe))));
}

// a * c (not renormalised: lo may reach a few units in the last place of hi)
__device__ __forceinline__ ff ff_mul(ff a, ff c) {
  const float p = __fmul_rn(a.h, c.h);
  const float e = fmaf(a.h, c.h, -p);
  return {p, fmaf(a.h, c.l, fmaf(a.l, c.h, e))};
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const ff s = two_sum(a.h, b.h);
  return {s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l))};
}

__device__ __forceinline__ ff ff_neg(ff a) { return {-a.h, -a.l}; }

// a - b to about 2^-47 of the difference itself, however close a and b are:
// both parts are subtracted exactly (two-sum), then renormalised.
__device__ __forceinline__ ff ff_diff(ff a, ff b) {
  const ff sh = two_sum(a.h, -b.h);
  const ff sl = two_sum(a.l, -b.l);
  const ff s = two_sum(sh.h, sl.h);
  return {s.h, __fadd_rn(s.l, __fadd_rn(sh.l, sl.l))};
}

}  // namespace ibg
