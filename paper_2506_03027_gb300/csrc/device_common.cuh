// device_common.cuh -- device helpers shared by the CUDA translation units of libcfs.
#pragma once

#include <cuda_runtime.h>

#include "cfs_internal.h"

namespace cfs {

__device__ __forceinline__ int wrapc(int i, int n) {
  int r = i % n;
  return r < 0 ? r + n : r;
}

// 1/x for FP64: hardware approximation refined by two Newton-Raphson steps r <- r + r (1 - x r)
// (Newton's method for the reciprocal; each step squares the relative error).  Within one ulp of
// the correctly rounded quotient for the positive normal densities it is used on.
__device__ __forceinline__ double recip(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}
__device__ __forceinline__ float recip(float x) { return 1.0f / x; }

// x^a = exp(a ln x) in FP64 for positive normal x (the viscosity law mu = T^a), with about 40
// FP64 operations.  ln x: reduction x = m 2^e with m in [1/sqrt(2), sqrt(2)) read off the bit
// fields, ln m = 2 atanh(s) with s = (m - 1)/(m + 1), |s| <= 0.1716, by the series
// sum s^(2j+1)/(2j+1) to s^23.  exp y: reduction y = k ln 2 + r, |r| <= ln(2)/2, with ln 2 split
// into a head of 32 significant bits and the tail (Cody and Waite's reduction: k ln2_head is
// exact), the Taylor series of exp r to r^14/14!, and 2^k added to the exponent field.  The split
// constants: the head is the double nearest ln 2 with its low 21 mantissa bits cleared, the tail
// ln 2 - head rounded (from a 60-digit ln 2).  Relative error below 4.5e-16 (1 + |a ln x|): the
// rounding of a ln x passes into the result.  Any other x (zero, subnormal, negative, infinite,
// NaN), or |a ln x| >= 700, goes to the library's pow.
__device__ __forceinline__ double pow_pos(double x, double a) {
  if (!(x >= 2.2250738585072014e-308) || !(x <= 1.7976931348623157e308)) return pow(x, a);
  const int hi = __double2hiint(x);
  int e = ((hi >> 20) & 0x7ff) - 1023;
  double m = __hiloint2double((hi & 0x000fffff) | 0x3ff00000, __double2loint(x));  // [1, 2)
  if (m > 1.4142135623730951) {
    m *= 0.5;
    e += 1;
  }
  const double s = (m - 1.0) * recip(m + 1.0);
  const double s2 = s * s;
  double p = 1.0 / 23.0;
  p = fma(p, s2, 1.0 / 21.0);
  p = fma(p, s2, 1.0 / 19.0);
  p = fma(p, s2, 1.0 / 17.0);
  p = fma(p, s2, 1.0 / 15.0);
  p = fma(p, s2, 1.0 / 13.0);
  p = fma(p, s2, 1.0 / 11.0);
  p = fma(p, s2, 1.0 / 9.0);
  p = fma(p, s2, 1.0 / 7.0);
  p = fma(p, s2, 1.0 / 5.0);
  p = fma(p, s2, 1.0 / 3.0);
  const double lnm = 2.0 * s * fma(p, s2, 1.0);
  const double LN2_HEAD = 0.6931471803691238, LN2_TAIL = 1.9082149292705877e-10;
  const double ed = (double)e;
  // a ln x = a (e ln2_head + (e ln2_tail + ln m)); e ln2_head is exact (32 + 11 bits)
  const double y = a * fma(ed, LN2_HEAD, fma(ed, LN2_TAIL, lnm));
  if (!(fabs(y) < 700.0)) return pow(x, a);  // 2^k must stay in the normal range
  // k = nearest integer of y / ln 2
  const double kd = rint(y * 1.4426950408889634);
  double r = fma(-kd, LN2_HEAD, y);
  r = fma(-kd, LN2_TAIL, r);
  double q = 1.0 / 87178291200.0;  // 1/14!
  q = fma(q, r, 1.0 / 6227020800.0);
  q = fma(q, r, 1.0 / 479001600.0);
  q = fma(q, r, 1.0 / 39916800.0);
  q = fma(q, r, 1.0 / 3628800.0);
  q = fma(q, r, 1.0 / 362880.0);
  q = fma(q, r, 1.0 / 40320.0);
  q = fma(q, r, 1.0 / 5040.0);
  q = fma(q, r, 1.0 / 720.0);
  q = fma(q, r, 1.0 / 120.0);
  q = fma(q, r, 1.0 / 24.0);
  q = fma(q, r, 1.0 / 6.0);
  q = fma(q, r, 0.5);
  q = fma(q, r, 1.0);
  q = fma(q, r, 1.0);
  const int k = (int)kd;
  return __hiloint2double(__double2hiint(q) + (k << 20), __double2loint(q));
}

// ---- FP64 <-> FP32 conversions on the integer pipe
// On this GPU conversions between FP64 and FP32 issue on the FP64 pipe, which runs at 1/64 of the
// FP32 rate; the FP32-intermediate form converts every stencil point, so these do it with integer
// operations on the IEEE-754 binary64 / binary32 bit fields instead.

// FP64 -> FP32, rounded to nearest with ties away from zero (differs from round-to-nearest-even
// only on exact ties).  |x| < 2^-126 gives a signed zero; |x| >= 2^128, inf and NaN give NaN.
// The 23 kept mantissa bits and the low 8 bits of the 11-bit exponent are bits 0..30 of
// (hi << 3 | lo >> 29); the exponent rebias 1023 -> 127 (minus 896 = 3.5 * 256) is a flip of the
// top bit of that 8-bit field for every exponent in the FP32 normal range.
__device__ __forceinline__ float d2f_fast(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned ahi = hi & 0x7fffffffu;
  unsigned t = __funnelshift_l(lo, hi, 3);
  t = ((t & 0x7fffffffu) ^ 0x40000000u) + ((lo >> 28) & 1u);  // a mantissa carry bumps the exponent
  t = (ahi < 0x38100000u) ? 0u : t;
  t = (ahi >= 0x47f00000u) ? 0x7fc00000u : t;
  return __uint_as_float(t | (hi & 0x80000000u));
}

// FP32 -> FP64, exact for normal numbers; zero and subnormals give a signed zero, inf and NaN give
// NaN.  The exponent rebias 127 -> 1023 adds 896 << 20 to the high word.
__device__ __forceinline__ double f2d_fast(float f) {
  const unsigned b = __float_as_uint(f), ab = b & 0x7fffffffu;
  unsigned hi = ((ab >> 3) + 0x38000000u) | (b & 0x80000000u);
  unsigned lo = b << 29;
  if (ab < 0x00800000u) { hi = b & 0x80000000u; lo = 0u; }
  if (ab >= 0x7f800000u) { hi = 0x7ff80000u; lo = 0u; }
  return __hiloint2double((int)hi, (int)lo);
}

// x - ref in FP32 with the accuracy of the FP64 difference rounded once more: x = h + e with h
// the FP32 truncation of x (exact) and e the remaining 29 mantissa bits scaled by 2^(E-1075);
// ref = rh + rl given as two floats.  (h - rh) is exact when x and ref are within a factor of two
// (Sterbenz), so the deviation keeps full FP32 precision however small it is relative to x.
__device__ __forceinline__ float dev_fast(double x, float rh, float rl) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned ahi = hi & 0x7fffffffu, e = ahi >> 20;
  unsigned t = (__funnelshift_l(lo, hi, 3) & 0x7fffffffu) ^ 0x40000000u;
  t = (ahi < 0x38100000u) ? 0u : t;
  t = (ahi >= 0x47f00000u) ? 0x7fc00000u : t;
  const float h = __uint_as_float(t | (hi & 0x80000000u));
  // remainder m 2^(E-1075), m = lo & (2^29 - 1), in FP32 arithmetic only: its top 23 and bottom 6
  // bits become exact floats by writing them as the mantissa under a power of two 2^k and
  // subtracting 2^k; the sum of the two rounds once.  Zero when 2^(E-1052) is not a normal float.
  const unsigned m = lo & 0x1fffffffu;
  const unsigned eb1 = (e - 919u) << 23, eb2 = (e - 925u) << 23;  // 2^(E-1046), 2^(E-1052)
  float r = (__uint_as_float(eb1 | (m >> 6)) - __uint_as_float(eb1)) +
            (__uint_as_float(eb2 | (m & 63u)) - __uint_as_float(eb2));
  r = (e >= 926u) ? r : 0.f;
  r = (hi & 0x80000000u) ? -r : r;
  return (h - rh) + (r - rl);
}

// Asynchronous global -> shared copies (cp.async; completion by cp_async_wait_all + a barrier).
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Delay of face f (0..5) of sub-domain sid at this step, clamped so every level exists.
__device__ __forceinline__ int face_delay(const StepSched& sc, int sid, int f) {
  int k = 0;
  if (sc.algo == 1) k = (int)((sc.n - sc.C) % sc.L);
  else if (sc.algo == 2) k = sc.table[sid * 6 + f];
  if (k > sc.cap) k = (int)sc.cap;
  if (k < 0) k = 0;
  return k;
}

// In graph mode the step index comes from device memory; derive what depends on it.
__device__ __forceinline__ StepSched resolve(StepSched sc) {
  if (sc.dn) {
    const long long n = *sc.dn;
    sc.n = n;
    sc.cap = n - sc.C + 1;
    sc.mode = (sc.algo == 0 || n < sc.C) ? 0 : (sc.at ? 1 : 2);
    sc.table = (sc.algo == 2 && sc.table_base) ? sc.table_base + n * (long long)sc.nsub * 6 : nullptr;
  }
  return sc;
}

// Ring level n (plus = 0) or n + 1 (plus = 1) when flagged, otherwise the given buffer.
__device__ __forceinline__ const double* ring_or(const double* p, int flag, const double* ring, const StepSched& sc,
                                                 int plus) {
  return flag ? ring + (long long)((sc.n + plus) % sc.R) * 5 * sc.Ntot : p;
}

}  // namespace cfs
