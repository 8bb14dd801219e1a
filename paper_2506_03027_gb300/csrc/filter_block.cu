// filter_block.cu -- the tenth-order Pade filter (Sec. 2) of the FP32-intermediate form on
// asynchronous (AT / AS) steps: all three passes of one sub-domain and one conserved variable in
// one CTA.
//
// On an asynchronous step the halo of every pass comes from the ring of delayed levels
// (AT: extrapolation to t_{n+1} with the weights c(k+1), in FP64; AS: the latest visible level),
// not from the neighbours' previous pass, so a sub-domain can be filtered x -> y -> z on its own.
// The CTA keeps the sub-domain's values as FP32 deviations from a reference value of the
// sub-domain in shared memory (rows of odd stride: the lines of every pass are read without
// bank conflicts), solves each line's tridiagonal system for the increment with the same
// right side and Thomas factors as the per-pass kernels (Dirichlet closure: zero increment at
// the first halo point), adds the increments in FP32 between passes, and writes
// U + (w_final - w_initial) in FP64 once.  The state is read and written once per step instead of
// once per pass.  Synchronous steps keep the per-pass kernels (their halo is the neighbours'
// previous pass).  The halo values -- 10 per line and pass, each a C-level FP64 sum over the
// ring -- come from k_filter_block_halo, which runs just before with one thread per value (many
// warps per SM hide the ring reads that a 512-thread, 176-KB CTA cannot) and stores them as FP32
// deviations for coalesced loads.
#include <cuda_runtime.h>

#include <mutex>

#include "cfs_internal.h"
#include "device_common.cuh"

namespace cfs {

namespace {

constexpr int FB_THREADS = 512;

__host__ __device__ constexpr int fb_row(int n) { return n | 1; }

template <int N>
__host__ __device__ inline size_t fb_smem(void) {
  return sizeof(float) * ((size_t)fb_row(N) * N * N + 2 * N + 10 * (N * N + 1));
}

// The halos of one (sub-domain, variable, pass): 5 points beyond each end of every line, from the
// ring (wrapped in the block): AT the extrapolation to t_{n+1} with the weights c(k+1) of the C
// delayed levels in FP64, AS the latest visible level; stored as FP32 deviations from the
// sub-domain's reference value (its first own value of the filter input), [10][N * N] per pass.
// Items are ordered so that consecutive threads read consecutive points: h fastest for the x pass
// (the 5 points of an end are adjacent in x), the line (x fastest) otherwise.
template <int N>
__global__ void __launch_bounds__(256) k_filter_block_halo(Geometry g, StepSched sc, FilterBlockLaunch f) {
  sc = resolve(sc);
  if (sc.mode == 0) return;  // synchronous step: the per-pass kernels filter it
  const double* __restrict__ Uin = ring_or(f.Uin, f.in_ring, f.ring, sc, 0);
  const int b = blockIdx.x;  // (sub-domain, variable, axis); the CTA loops over its 10 N^2 values
  const int sid = b / 15, var = (b / 3) % 5, axis = b % 3;
  const SubDev d = f.subs[sid];
  const long long plane = (long long)d.bnx * d.bny;
  const long long vbase = d.bbase + (long long)var * d.bN;
  const long long lvN = 5 * g.N;
  const long long own0 = (long long)d.ox + (long long)d.bnx * d.oy + plane * d.oz;
  const double ref = Uin[vbase + own0];
  const float rh = d2f_fast(ref), rl = dev_fast(ref, rh, 0.f);
  // strides along the pass axis and the two line axes (x fastest), the wrap length along the axis
  const long long sA = axis == 0 ? 1 : (axis == 1 ? (long long)d.bnx : plane);
  const long long s1 = axis == 0 ? (long long)d.bnx : 1, s2 = axis == 2 ? (long long)d.bnx : plane;
  const int nA = axis == 0 ? d.bnx : (axis == 1 ? d.bny : d.bnz);
  const int oA = axis == 0 ? d.ox : (axis == 1 ? d.oy : d.oz);
  const long long base12 = vbase + own0 - (long long)oA * sA;  // origin of the lines, axis coordinate 0
  const int nlev = sc.mode == 2 ? 1 : sc.C;
  // per end of the lines: ring-level offsets of the C delayed levels (slot (n mod R) - k - l,
  // wrapped once) and their weights c(k + 1)
  long long lev[2][CFS_MAX_LEVELS];
  double wf[2][CFS_MAX_LEVELS];
  const int nR = (int)(sc.n % sc.R);
#pragma unroll
  for (int sd = 0; sd < 2; ++sd) {
    const int kd = face_delay(sc, sid, 2 * axis + sd);
#pragma unroll
    for (int lv = 0; lv < CFS_MAX_LEVELS; ++lv) {
      int q = nR - kd - lv;
      q = q < 0 ? q + sc.R : q;
      lev[sd][lv] = lv < nlev ? (long long)q * lvN : 0;
      wf[sd][lv] = sc.mode == 2 ? 1.0 : (lv < nlev ? __ldg(sc.Wf + kd * sc.C + lv) : 0.0);
    }
  }
  float* __restrict__ out = f.halo + (long long)b * 10 * N * N;
#pragma unroll 4
  for (int e = threadIdx.x; e < 10 * N * N; e += blockDim.x) {
    const int h = axis == 0 ? e % 10 : e / (N * N), l = axis == 0 ? e / 10 : e % (N * N);
    const int t1 = l % N, t2 = l / N;
    const int sd = h < 5 ? 0 : 1;
    int ca = oA + (h < 5 ? h - 5 : N + h - 5);
    ca = ca < 0 ? ca + nA : (ca >= nA ? ca - nA : ca);
    const long long gi = base12 + t1 * s1 + t2 * s2 + ca * sA;
    double r[CFS_MAX_LEVELS];
#pragma unroll
    for (int lv = 0; lv < CFS_MAX_LEVELS; ++lv) r[lv] = lv < nlev ? f.ring[(sd ? lev[1][lv] : lev[0][lv]) + gi] : 0.0;
    double v = 0.0;
#pragma unroll
    for (int lv = 0; lv < CFS_MAX_LEVELS; ++lv)
      if (lv < nlev) v = fma(sd ? wf[1][lv] : wf[0][lv], r[lv], v);
    out[h * (N * N) + l] = dev_fast(v, rh, rl);
  }
}

template <int N>
__global__ void __launch_bounds__(FB_THREADS, 1) k_filter_block(Geometry g, StepSched sc, FilterBlockLaunch f) {
  sc = resolve(sc);
  if (sc.mode == 0) return;  // synchronous step: the per-pass kernels filter it
  const double* __restrict__ Uin = ring_or(f.Uin, f.in_ring, f.ring, sc, 0);
  double* __restrict__ Uout = const_cast<double*>(ring_or(f.Uout, f.out_ring, f.ring, sc, 1));
  constexpr int RX = fb_row(N), RXY = RX * N;
  const int sid = blockIdx.x / 5, var = blockIdx.x % 5;
  const SubDev d = f.subs[sid];
  extern __shared__ __align__(16) float fbs[];
  float* blk = fbs;                   // [N][N][RX]: deviations, x fastest
  float* sTh = fbs + (size_t)RXY * N;  // cp[N], im[N]
  float* sHalo = sTh + 2 * N;          // [10][N * N + 1]: the halo deviations of every line of a pass
  const int tid = threadIdx.x;
  const long long plane = (long long)d.bnx * d.bny;
  const long long vbase = d.bbase + (long long)var * d.bN;
  const double* __restrict__ U = Uin + vbase;
  double* __restrict__ Uo = Uout + vbase;
  const long long own0 = (long long)d.ox + (long long)d.bnx * d.oy + plane * d.oz;
  const double ref = U[own0];
  const float rh = d2f_fast(ref), rl = dev_fast(ref, rh, 0.f);
  // Thomas factors of a line of N points (the same on every axis)
  for (int t = tid; t < 2 * N; t += FB_THREADS) {
    const double* cp = f.thomas + (long long)N * 2 * f.Lmax;
    sTh[t] = (float)(t < N ? cp[t] : cp[f.Lmax + t - N]);
  }
  // ---- load the own values as deviations (unrolled: several loads in flight per thread)
#pragma unroll 8
  for (int q = tid; q < N * N * N; q += FB_THREADS) {
    const int x = q % N, y = (q / N) % N, z = q / (N * N);
    const long long gi = own0 + x + (long long)d.bnx * y + plane * z;
    blk[z * RXY + y * RX + x] = dev_fast(__ldg(U + gi), rh, rl);
  }
  __syncthreads();
  const float b1 = (float)f.b1, al = (float)f.alpha;
  float hm[6];
#pragma unroll
  for (int m = 2; m <= 5; ++m) hm[m] = (float)f.h[m];
  const float* cpf = sTh;
  const float* imf = sTh + N;
#pragma unroll
  for (int axis = 0; axis < 3; ++axis) {
    const int f1 = axis == 0 ? 1 : 0, f2 = axis == 2 ? 1 : 2;
    const int st[3] = {1, RX, RXY};
    const int sa = st[axis];
    // ---- halo: the pass's 10 x N^2 values from k_filter_block_halo (coalesced)
    const float* __restrict__ hsrc = f.halo + ((long long)blockIdx.x * 3 + axis) * 10 * N * N;
#pragma unroll 4
    for (int e = tid; e < 10 * N * N; e += FB_THREADS) {
      const int h = e / (N * N), l = e % (N * N);
      sHalo[h * (N * N + 1) + l] = __ldg(hsrc + e);
    }
    __syncthreads();
#pragma unroll 1
    for (int l = tid; l < N * N; l += FB_THREADS) {
      const int t1 = l % N, t2 = l / N;
      const int base = t1 * st[f1] + t2 * st[f2];
      float w[N + 10];
#pragma unroll
      for (int i = 0; i < N; ++i) w[i + 5] = blk[base + i * sa];
#pragma unroll
      for (int h = 0; h < 5; ++h) {
        w[h] = sHalo[h * (N * N + 1) + l];
        w[N + 5 + h] = sHalo[(5 + h) * (N * N + 1) + l];
      }
      // right side sum_n (a_n/2)(f_{i+n} + f_{i-n}) - (alpha f_{i-1} + f_i + alpha f_{i+1}), written
      // as second differences; forward elimination
      float dd[N];
      float dprev = 0.f;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const float c2 = 2.f * w[i + 5];
        float rhs = b1 * ((w[i + 6] + w[i + 4]) - c2);
#pragma unroll
        for (int m = 2; m <= 5; ++m) rhs = fmaf(hm[m], (w[i + 5 + m] + w[i + 5 - m]) - c2, rhs);
        const float dc = (i == 0 ? rhs : fmaf(-al, dprev, rhs)) * imf[i];
        dd[i] = dc;
        dprev = dc;
      }
      // back substitution; the filtered deviation replaces the value
      float xn = dprev;
      blk[base + (N - 1) * sa] = w[N + 4] + xn;
#pragma unroll
      for (int i = N - 2; i >= 0; --i) {
        const float x = fmaf(-cpf[i], xn, dd[i]);
        blk[base + i * sa] = w[i + 5] + x;
        xn = x;
      }
    }
    __syncthreads();
  }
  // ---- U + (filtered - initial deviation), in FP64
#pragma unroll 8
  for (int q = tid; q < N * N * N; q += FB_THREADS) {
    const int x = q % N, y = (q / N) % N, z = q / (N * N);
    const long long gi = own0 + x + (long long)d.bnx * y + plane * z;
    const double u = __ldg(U + gi);
    Uo[gi] = u + f2d_fast(blk[z * RXY + y * RX + x] - dev_fast(u, rh, rl));
  }
}

// The shared-memory opt-in is a per-device attribute: set once on every device that launches.
template <int N>
int fb_prepare() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return (int)e;
  if (dev < 0 || dev >= 64) return (int)cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev]) return 0;
  e = cudaFuncSetAttribute(k_filter_block<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fb_smem<N>());
  if (e == cudaSuccess) done[dev] = true;
  return (int)e;
}

}  // namespace

bool filter_block_supported(int n) { return n == 16 || n == 32; }

int launch_filter_block(const Geometry& g, const StepSched& sc, const FilterBlockLaunch& f, int n, void* stream,
                        long long* launches, const Timer* tm) {
  cudaStream_t st = (cudaStream_t)stream;
  int rc = n == 32 ? fb_prepare<32>() : fb_prepare<16>();
  if (rc) return rc;
  if (tm) tm->rec(tm->self, 3, 1);
  const unsigned nb = (unsigned)(5 * f.nsub);
  if (n == 32) {
    k_filter_block_halo<32><<<(unsigned)(15 * f.nsub), 256, 0, st>>>(g, sc, f);
    k_filter_block<32><<<nb, FB_THREADS, fb_smem<32>(), st>>>(g, sc, f);
  } else {
    k_filter_block_halo<16><<<(unsigned)(15 * f.nsub), 256, 0, st>>>(g, sc, f);
    k_filter_block<16><<<nb, FB_THREADS, fb_smem<16>(), st>>>(g, sc, f);
  }
  if (tm) tm->rec(tm->self, 3, 0);
  if (launches) *launches += 2;
  return (int)cudaGetLastError();
}

}  // namespace cfs
