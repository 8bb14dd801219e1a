// noalloc.cu -- cfs_diagnostics_static: the diagnostics reduction for callers that must not
// allocate device memory.
//
// Some callers cannot call cudaMalloc: an in-situ monitoring hook running inside a larger
// simulation whose own pool allocator already owns the GPU's memory, or a time-critical loop in
// which an allocation (which may synchronise the device) is not allowed.  This entry point
// computes the same quantities as cfs_diagnostics on a state the caller holds in device memory,
// with its only scratch (the per-block partial sums) in a fixed array compiled into the library.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "cfs.h"
#include "device_common.cuh"

namespace {

constexpr int kThreads = 256;
// One block reduces 256 points into 8 partial sums; the array holds CFS_DIAG_STATIC_MAX_POINTS /
// 256 blocks of partials (4 MiB).  Every GPU that loads the library keeps this array until exit.
constexpr long long kMaxBlocks = CFS_DIAG_STATIC_MAX_POINTS / kThreads;
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_partials[kMaxBlocks * 8];

std::mutex g_mu;
double* g_dev_ptr[kMaxDevices] = {nullptr};

struct Grid {
  int nx, ny, nz, ndim, r;
  long long N;
  double c1[3], c2[3], dV;
};

__device__ __forceinline__ int wrap(int i, int n) {
  int r = i % n;
  return r < 0 ? r + n : r;
}

// Two velocity components (c0, c1) of the point (x, y, z), periodic wrap: one reciprocal of the
// density (Newton-refined) per stencil point instead of a division per component.
__device__ __forceinline__ void vel2(const double* U, const Grid& g, int x, int y, int z, int c0, int c1, double* a,
                                     double* b) {
  const long long i = (long long)wrap(x, g.nx) + (long long)g.nx * ((long long)wrap(y, g.ny) + (long long)g.ny * wrap(z, g.nz));
  const double ir = cfs::recip(U[i]);
  *a = U[(1 + c0) * g.N + i] * ir;
  *b = U[(1 + c1) * g.N + i] * ir;
}

// One point per thread; block b writes its 8 partial sums to partials[8 b .. 8 b + 7].
__global__ void __launch_bounds__(kThreads) k_diag_blocks(Grid g, const double* __restrict__ U,
                                                           double* __restrict__ partials) {
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  const long long i = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (i < g.N) {
    const int x = (int)(i % g.nx), y = (int)((i / g.nx) % g.ny), z = (int)(i / ((long long)g.nx * g.ny));
    double u[5];
    for (int v = 0; v < 5; ++v) {
      u[v] = U[v * g.N + i];
      if (!isfinite(u[v])) acc[7] = 1.0;
      acc[2 + v] = u[v] * g.dV;
    }
    const double rho = u[0], ir = cfs::recip(rho), vx = u[1] * ir, vy = u[2] * ir, vz = u[3] * ir;
    acc[0] = 0.5 * rho * (vx * vx + vy * vy + vz * vz);
    // the vorticity needs d v_c / d x_a for c != a only: along axis a, the two other components
    double dv[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a >= g.ndim) break;
      const int c0 = a == 0 ? 1 : 0, c1 = a == 2 ? 1 : 2;
      const int ex = a == 0, ey = a == 1, ez = a == 2;
      double p0, p1, m0, m1;
      vel2(U, g, x + ex, y + ey, z + ez, c0, c1, &p0, &p1);
      vel2(U, g, x - ex, y - ey, z - ez, c0, c1, &m0, &m1);
      double d0 = g.c1[a] * (p0 - m0), d1 = g.c1[a] * (p1 - m1);
      if (g.r == 2) {
        vel2(U, g, x + 2 * ex, y + 2 * ey, z + 2 * ez, c0, c1, &p0, &p1);
        vel2(U, g, x - 2 * ex, y - 2 * ey, z - 2 * ez, c0, c1, &m0, &m1);
        d0 += g.c2[a] * (p0 - m0);
        d1 += g.c2[a] * (p1 - m1);
      }
      dv[c0][a] = d0;
      dv[c1][a] = d1;
    }
    const double wx = dv[2][1] - dv[1][2], wy = dv[0][2] - dv[2][0], wz = dv[1][0] - dv[0][1];
    acc[1] = 0.5 * rho * (wx * wx + wy * wy + wz * wz);
  }
  __shared__ double sh[8][kThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int c = 0; c < 8; ++c) {
    double v = acc[c];
    for (int o = 16; o > 0; o >>= 1) {
      const double other = __shfl_down_sync(0xffffffffu, v, o);
      v = (c == 7) ? fmax(v, other) : v + other;
    }
    if (lane == 0) sh[c][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < 8) {
    const int c = threadIdx.x;
    double v = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) v = (c == 7) ? fmax(v, sh[c][w]) : v + sh[c][w];
    partials[(long long)blockIdx.x * 8 + c] = v;
  }
}

// Fixed-order second pass, one warp per quantity (8 warps): lane l sums the partials of blocks
// l, l + 32, l + 64, ... in block order, then the 32 lane sums combine in a fixed shuffle tree.
// The order depends only on the number of blocks, so the result is deterministic.
__global__ void __launch_bounds__(256) k_diag_blocks_final(const double* __restrict__ partials, long long nblocks,
                                                           long long N, double* __restrict__ out) {
  const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double v = 0.0;
  for (long long b = lane; b < nblocks; b += 32) v = (c == 7) ? fmax(v, partials[b * 8 + c]) : v + partials[b * 8 + c];
  for (int o = 16; o > 0; o >>= 1) {
    const double other = __shfl_down_sync(0xffffffffu, v, o);
    v = (c == 7) ? fmax(v, other) : v + other;
  }
  if (lane == 0) out[c] = (c < 2) ? v / (double)N : v;
}

void put(char* err, size_t len, const char* msg) {
  if (err && len) std::snprintf(err, len, "%s", msg);
}

}  // namespace

extern "C" cfs_status cfs_diagnostics_static(const double* U, int nx, int ny, int nz, const double* spacing, int order,
                                             double* out, void* cuda_stream, char* err, size_t err_len) {
  if (!U || !out || !spacing) {
    put(err, err_len, "cfs_diagnostics_static: null pointer");
    return CFS_EINVAL;
  }
  if (nx < 1 || ny < 1 || nz < 1 || (order != 2 && order != 4)) {
    put(err, err_len, "cfs_diagnostics_static: bad grid size or order");
    return CFS_EINVAL;
  }
  const long long N = (long long)nx * ny * nz;
  if (N > CFS_DIAG_STATIC_MAX_POINTS) {
    char msg[160];
    std::snprintf(msg, sizeof(msg),
                  "cfs_diagnostics_static: %lld points exceed the static scratch limit of %lld points",
                  N, (long long)CFS_DIAG_STATIC_MAX_POINTS);
    put(err, err_len, msg);
    return CFS_EINVAL;
  }
  for (int a = 0; a < 3; ++a)
    if (!(spacing[a] > 0.0)) {
      put(err, err_len, "cfs_diagnostics_static: spacing must be positive");
      return CFS_EINVAL;
    }
  // Set-up, once per device: the array's name is only a host-side stand-in, so look up its
  // device address with that device current.
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    put(err, err_len, "cfs_diagnostics_static: no usable CUDA device");
    return CFS_ECUDA;
  }
  double* partials = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_dev_ptr[dev]) {
      e = cudaGetSymbolAddress((void**)&g_dev_ptr[dev], g_partials);
      if (e != cudaSuccess) {
        g_dev_ptr[dev] = nullptr;
        put(err, err_len, cudaGetErrorString(e));
        return CFS_ECUDA;
      }
    }
    partials = g_dev_ptr[dev];
  }
  Grid g{};
  g.nx = nx; g.ny = ny; g.nz = nz; g.N = N;
  g.ndim = nz > 1 ? 3 : 2;
  g.r = order == 4 ? 2 : 1;
  const double a = order == 4 ? 4.0 / 3.0 : 1.0, b = order == 4 ? -1.0 / 3.0 : 0.0;
  for (int k = 0; k < 3; ++k) {
    g.c1[k] = (a / 2.0) / spacing[k];
    g.c2[k] = (b / 4.0) / spacing[k];
  }
  g.dV = spacing[0] * spacing[1] * (g.ndim == 3 ? spacing[2] : 1.0);
  const long long nblocks = (N + kThreads - 1) / kThreads;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  k_diag_blocks<<<(unsigned)nblocks, kThreads, 0, st>>>(g, U, partials);
  k_diag_blocks_final<<<1, 256, 0, st>>>(partials, nblocks, N, out);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    put(err, err_len, cudaGetErrorString(e));
    return CFS_ECUDA;
  }
  return CFS_OK;
}
