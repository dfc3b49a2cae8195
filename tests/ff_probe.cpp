// Host test driver for the double-FP32 helpers of csrc/ff.cuh: the device
// intrinsics they use are given host definitions with the same IEEE-754
// semantics (round to nearest even, no contraction: build with
// -ffp-contract=off), then seeded random inputs are checked against long
// double arithmetic.  Prints one line per property: name, cases, failures.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>

#define __device__
#define __forceinline__ inline

static inline float __uint_as_float(unsigned u) { float f; std::memcpy(&f, &u, 4); return f; }
static inline unsigned __float_as_uint(float f) { unsigned u; std::memcpy(&u, &f, 4); return u; }
static inline float __int_as_float(int i) { float f; std::memcpy(&f, &i, 4); return f; }
static inline int __double2hiint(double x) { uint64_t u; std::memcpy(&u, &x, 8); return int(uint32_t(u >> 32)); }
static inline int __double2loint(double x) { uint64_t u; std::memcpy(&u, &x, 8); return int(uint32_t(u)); }
static inline double __hiloint2double(int hi, int lo) {
  const uint64_t u = (uint64_t(uint32_t(hi)) << 32) | uint32_t(lo);
  double x;
  std::memcpy(&x, &u, 8);
  return x;
}
static inline float __double2float_rn(double x) { return float(x); }
static inline float __fadd_rn(float a, float b) { volatile float r = a + b; return r; }
static inline float __fsub_rn(float a, float b) { volatile float r = a - b; return r; }
static inline float __fmul_rn(float a, float b) { volatile float r = a * b; return r; }

#include "ff.cuh"

using namespace ibg;

static uint64_t state = 0x9E3779B97F4A7C15ULL;
static uint64_t next() {   // xorshift64*
  state ^= state >> 12;
  state ^= state << 25;
  state ^= state >> 27;
  return state * 2685821657736338717ULL;
}
static double unit() { return double(next() >> 11) * (1.0 / 9007199254740992.0); }
// a double with a random sign, full random mantissa and exponent in [e0, e1]
static double rnd(int e0, int e1) {
  const double m = 1.0 + unit();
  const int e = e0 + int(next() % uint64_t(e1 - e0 + 1));
  return (next() & 1 ? -1.0 : 1.0) * std::ldexp(m, e);
}

static void report(const char* name, long n, long bad) { std::printf("%s %ld %ld\n", name, n, bad); }

int main() {
  const long N = 200000;
  // 1. dsplit: hi is x cut to 24 bits, hi + lo within 2^-48 |x| (|x| >= 2^-100)
  long bad = 0;
  for (long i = 0; i < N; ++i) {
    const double x = rnd(-100, 100);
    const ff s = dsplit(x);
    const long double sum = (long double)s.h + (long double)s.l;
    const bool trunc = std::fabs(double(s.h)) <= std::fabs(x) && std::signbit(s.h) == std::signbit(x) &&
                       std::fabs(x - double(s.h)) < std::ldexp(std::fabs(x), -22);
    if (!trunc || std::fabs((long double)x - sum) > std::ldexp((long double)std::fabs(x), -48)) ++bad;
  }
  report("dsplit", N, bad);
  // tiny values read as zero; near the bottom of the FP32 range hi + lo stays
  // within 2^-149 of x
  bad = 0;
  if (dsplit(1e-40).h != 0.f || dsplit(-0.0).h != 0.f || dsplit(0.0).l != 0.f) ++bad;
  {
    const double x = std::ldexp(1.0 + unit(), -120);
    const ff s = dsplit(x);
    if (std::fabs((long double)x - ((long double)s.h + s.l)) > std::ldexp(1.0L, -149)) ++bad;
  }
  report("dsplit_edges", 3, bad);
  // 2. f2d is the exact conversion
  bad = 0;
  for (long i = 0; i < N; ++i) {
    const float f = __uint_as_float(uint32_t(next()));
    if (std::isnan(f)) continue;
    if (f2d(f) != double(f) || std::signbit(f2d(f)) != std::signbit(f)) ++bad;
  }
  if (f2d(-0.f) != 0.0 || !std::signbit(f2d(-0.f))) ++bad;
  report("f2d", N + 1, bad);
  // 3. wf: exact small integers
  bad = 0;
  for (int w = -4096; w <= 4096; ++w)
    if (wf(w) != float(w)) ++bad;
  report("wf", 8193, bad);
  // 4. two_sum is error-free
  bad = 0;
  for (long i = 0; i < N; ++i) {
    const float a = float(rnd(-20, 20)), b = float(rnd(-20, 20));
    const ff s = two_sum(a, b);
    if ((long double)s.h + (long double)s.l != (long double)a + (long double)b) ++bad;
  }
  report("two_sum", N, bad);
  // 5. an integer-weighted sum of 15 FP64 values (the mass stencil) within
  //    2^-44 of the sum of the terms' magnitudes
  bad = 0;
  long double worst = 0;
  for (long i = 0; i < N / 10; ++i) {
    ff acc{0.f, 0.f};
    long double ref = 0, mag = 0;
    const int e = -10 + int(next() % 20);
    for (int k = 0; k < 15; ++k) {
      const int w = int(next() % 25) - 4;
      const double x = rnd(e - 3, e + 3);
      ff_madd_int(acc, wf(w), dsplit(x));
      ref += (long double)w * x;
      mag += std::fabs((long double)w * x);
    }
    const long double err = std::fabs((long double)ff2d(acc) - ref) / mag;
    if (err > worst) worst = err;
    if (err > std::ldexp(1.0L, -44)) ++bad;
  }
  report("madd_int", N / 10, bad);
  std::fprintf(stderr, "madd_int worst relative error 2^%.2f\n", double(std::log2(worst)));
  // 6. ff_diff of nearby values keeps 2^-45 of the difference itself
  bad = 0;
  for (long i = 0; i < N; ++i) {
    const double x0 = rnd(-30, 30);
    const double xk = x0 * (1.0 + std::ldexp(unit() - 0.5, -int(next() % 40)));
    const ff a = dsplit(x0), b = dsplit(xk);
    const long double want = ((long double)a.h + a.l) - ((long double)b.h + b.l);
    const ff d = ff_diff(a, b);
    const long double got = (long double)d.h + (long double)d.l;
    if (std::fabs(got - want) > std::ldexp(std::fabs(want), -45) + 1e-300L) ++bad;
  }
  report("diff", N, bad);
  // 7. a pair times a pair constant, within 2^-44 of the product
  bad = 0;
  for (long i = 0; i < N; ++i) {
    const double x = rnd(-20, 20), c = rnd(-20, 20);
    const ff p = ff_mul(dsplit(x), dsplit(c));
    const long double want = (long double)x * (long double)c;
    if (std::fabs((long double)p.h + (long double)p.l - want) > std::ldexp(std::fabs(want), -44)) ++bad;
  }
  report("mul", N, bad);
  // 8. scale2 is ldexp; d2f rounds to the nearest FP32 number
  bad = 0;
  for (long i = 0; i < N; ++i) {
    const double x = rnd(-300, 300);
    const int sh = int(next() % 601) - 300;
    if (scale2(x, sh) != std::ldexp(x, sh)) ++bad;
  }
  if (scale2(0.0, 5) != 0.0 || scale2(1e-310, 3) != std::ldexp(1e-310, 3)) ++bad;
  report("scale2", N + 1, bad);
  bad = 0;
  for (long i = 0; i < N; ++i) {
    const double x = rnd(-100, 120);
    if (d2f(x) != float(x)) ++bad;
  }
  report("d2f", N, bad);
  return 0;
}
