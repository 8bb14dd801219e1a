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
