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

// x = h + r with h the FP32 truncation of x (exact) and r the remaining 29 mantissa bits scaled by
// 2^(E-1075), rounded once to FP32.  The range rules of d2f_fast hold for h; r is zero when
// 2^(E-1052) is not a normal float.
__device__ __forceinline__ void split_fast(double x, float& h, float& r) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned ahi = hi & 0x7fffffffu, e = ahi >> 20;
  unsigned t = (__funnelshift_l(lo, hi, 3) & 0x7fffffffu) ^ 0x40000000u;
  t = (ahi < 0x38100000u) ? 0u : t;
  t = (ahi >= 0x47f00000u) ? 0x7fc00000u : t;
  h = __uint_as_float(t | (hi & 0x80000000u));
  // m 2^(E-1075), m = lo & (2^29 - 1), in FP32 arithmetic only: its top 23 and bottom 6 bits become
  // exact floats by writing them as the mantissa under a power of two 2^k and subtracting 2^k;
  // the sum of the two rounds once.
  const unsigned m = lo & 0x1fffffffu;
  const unsigned eb1 = (e - 919u) << 23, eb2 = (e - 925u) << 23;  // 2^(E-1046), 2^(E-1052)
  float q = (__uint_as_float(eb1 | (m >> 6)) - __uint_as_float(eb1)) +
            (__uint_as_float(eb2 | (m & 63u)) - __uint_as_float(eb2));
  q = (e >= 926u) ? q : 0.f;
  r = (hi & 0x80000000u) ? -q : q;
}

// x - ref in FP32 with the accuracy of the FP64 difference rounded once more, ref = rh + rl given
// as two floats: (h - rh) is exact when x and ref are within a factor of two (Sterbenz), so the
// deviation keeps full FP32 precision however small it is relative to x.
__device__ __forceinline__ float dev_fast(double x, float rh, float rl) {
  float h, r;
  split_fast(x, h, r);
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

// One poll of an mbarrier phase (try_wait: may suspend the thread for a short time); true when the
// phase with the given parity has completed.
__device__ __forceinline__ bool mbar_poll(const unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"((unsigned)__cvta_generic_to_shared(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for an mbarrier phase: at most limit + 1 polls; false when it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(const unsigned long long* bar, unsigned parity, unsigned limit) {
  for (unsigned it = 0;; ++it) {
    if (mbar_poll(bar, parity)) return true;
    if (it >= limit) return false;
  }
}

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
