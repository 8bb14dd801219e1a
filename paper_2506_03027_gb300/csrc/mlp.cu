// mlp.cu -- the learned halo predictor's network: forward, backward and AdamW kernels.
//
// A 3-layer perceptron NIN -> NH -> NH -> NOUT with GELU activations (tanh form of Hendrycks &
// Gimpel) predicts, for one face column of a sub-domain's halo, the residual of the current-level
// halo values over the 3-level extrapolation (Eq. 14) from features of the delayed levels.
// Inputs are BF16, arithmetic FP32.  Each CTA processes a chunk of samples layer by layer as small
// GEMMs in shared memory; the weight gradients of a chunk are summed in a fixed order and the
// chunk partials reduced in chunk order, so training is deterministic.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <mutex>

#include <algorithm>

#include "cfs_internal.h"
#include "device_common.cuh"

namespace cfs {

namespace {

constexpr int S = 32;  // samples per CTA
constexpr int NT = 256;

__device__ __forceinline__ float gelu(float z) {
  const float k0 = 0.7978845608028654f, k1 = 0.044715f;  // sqrt(2/pi)
  return 0.5f * z * (1.f + tanhf(k0 * (z + k1 * z * z * z)));
}

__device__ __forceinline__ float gelu_grad(float z) {
  const float k0 = 0.7978845608028654f, k1 = 0.044715f;
  const float u = k0 * (z + k1 * z * z * z);
  const float t = tanhf(u);
  return 0.5f * (1.f + t) + 0.5f * z * (1.f - t * t) * k0 * (1.f + 3.f * k1 * z * z);
}

struct Smem {
  float w[MLP_NPARAM];
  float x[S][MLP_NIN + 1];
  float z1[S][MLP_NH], h1[S][MLP_NH], z2[S][MLP_NH], h2[S][MLP_NH], y[S][MLP_NOUT];
};

// dst[s][o] = act(b[o] + sum_i W[o][i] src[s][i]) for s < ns, with z (pre-activation) stored too
__device__ __forceinline__ void layer(const float* W, const float* b, const float* src, int ld_src, int nin, int nout,
                                      float* z, float* h, int ld_dst, int ns, bool act) {
  for (int e = threadIdx.x; e < ns * nout; e += NT) {
    const int s = e / nout, o = e % nout;
    float acc = b[o];
    const float* wr = W + o * nin;
    const float* xr = src + s * ld_src;
    for (int i = 0; i < nin; ++i) acc = fmaf(wr[i], xr[i], acc);
    if (z) z[s * ld_dst + o] = acc;
    h[s * ld_dst + o] = act ? gelu(acc) : acc;
  }
}

__device__ void load_chunk(Smem& sm, const float* __restrict__ params, const __nv_bfloat16* __restrict__ x, long long base,
                           int ns) {
  for (int p = threadIdx.x; p < MLP_NPARAM; p += NT) sm.w[p] = params[p];
  for (int e = threadIdx.x; e < ns * MLP_NIN; e += NT) {
    const int s = e / MLP_NIN, i = e % MLP_NIN;
    sm.x[s][i] = __bfloat162float(x[(base + s) * MLP_NIN + i]);
  }
  __syncthreads();
}

__device__ void forward_chunk(Smem& sm, int ns) {
  const float* W1 = sm.w + MLP_OFF_W1;
  const float* W2 = sm.w + MLP_OFF_W2;
  const float* W3 = sm.w + MLP_OFF_W3;
  layer(W1, sm.w + MLP_OFF_B1, &sm.x[0][0], MLP_NIN + 1, MLP_NIN, MLP_NH, &sm.z1[0][0], &sm.h1[0][0], MLP_NH, ns, true);
  __syncthreads();
  layer(W2, sm.w + MLP_OFF_B2, &sm.h1[0][0], MLP_NH, MLP_NH, MLP_NH, &sm.z2[0][0], &sm.h2[0][0], MLP_NH, ns, true);
  __syncthreads();
  layer(W3, sm.w + MLP_OFF_B3, &sm.h2[0][0], MLP_NH, MLP_NH, MLP_NOUT, nullptr, &sm.y[0][0], MLP_NOUT, ns, false);
  __syncthreads();
}

}  // namespace

__global__ void __launch_bounds__(NT) k_mlp_fwd(const float* __restrict__ params, const __nv_bfloat16* __restrict__ x,
                                                 float* __restrict__ y, long long nsamp) {
  extern __shared__ __align__(16) unsigned char raw[];
  Smem& sm = *reinterpret_cast<Smem*>(raw);
  for (long long base = (long long)blockIdx.x * S; base < nsamp; base += (long long)gridDim.x * S) {
    const int ns = (int)min((long long)S, nsamp - base);
    load_chunk(sm, params, x, base, ns);
    forward_chunk(sm, ns);
    for (int e = threadIdx.x; e < ns * MLP_NOUT; e += NT) y[base * MLP_NOUT + e] = sm.y[e / MLP_NOUT][e % MLP_NOUT];
    __syncthreads();
  }
}

// Mean-squared-error loss over all outputs of the batch; per chunk: forward, backward deltas,
// then the chunk's gradient partial[chunk][p] summed over its samples in order; loss partial too.
__global__ void __launch_bounds__(NT) k_mlp_bwd(const float* __restrict__ params, const __nv_bfloat16* __restrict__ x,
                                                 const float* __restrict__ target, long long nsamp, float* __restrict__ partial,
                                                 float* __restrict__ loss_partial) {
  extern __shared__ __align__(16) unsigned char raw[];
  Smem& sm = *reinterpret_cast<Smem*>(raw);
  const long long chunk = blockIdx.x;
  const long long base = chunk * S;
  if (base >= nsamp) return;
  const int ns = (int)min((long long)S, nsamp - base);
  load_chunk(sm, params, x, base, ns);
  forward_chunk(sm, ns);
  const float scale = 2.f / ((float)nsamp * MLP_NOUT);
  // dy (stored over y), loss
  __shared__ float red[NT];
  float lsum = 0.f;
  for (int e = threadIdx.x; e < ns * MLP_NOUT; e += NT) {
    const int s = e / MLP_NOUT, o = e % MLP_NOUT;
    const float d = sm.y[s][o] - target[(base + s) * MLP_NOUT + o];
    lsum += d * d;
    sm.y[s][o] = scale * d;
  }
  red[threadIdx.x] = lsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int i = 0; i < NT; ++i) t += red[i];
    loss_partial[chunk] = t;
  }
  const float* W2 = sm.w + MLP_OFF_W2;
  const float* W3 = sm.w + MLP_OFF_W3;
  // dz2 = (W3^T dy) * gelu'(z2), stored over h2's slot after it is used for dW3 below: keep h2,
  // write dz2 into z2
  for (int e = threadIdx.x; e < ns * MLP_NH; e += NT) {
    const int s = e / MLP_NH, i = e % MLP_NH;
    float acc = 0.f;
    for (int o = 0; o < MLP_NOUT; ++o) acc = fmaf(W3[o * MLP_NH + i], sm.y[s][o], acc);
    sm.z2[s][i] = acc * gelu_grad(sm.z2[s][i]);
  }
  __syncthreads();
  // dz1 = (W2^T dz2) * gelu'(z1), written into z1
  for (int e = threadIdx.x; e < ns * MLP_NH; e += NT) {
    const int s = e / MLP_NH, i = e % MLP_NH;
    float acc = 0.f;
    for (int o = 0; o < MLP_NH; ++o) acc = fmaf(W2[o * MLP_NH + i], sm.z2[s][o], acc);
    sm.z1[s][i] = acc * gelu_grad(sm.z1[s][i]);
  }
  __syncthreads();
  // parameter gradients of this chunk, summed over its samples in order
  float* out = partial + chunk * MLP_NPARAM;
  for (int p = threadIdx.x; p < MLP_NPARAM; p += NT) {
    float g = 0.f;
    if (p < MLP_OFF_B1) {  // W1[o][i]
      const int o = p / MLP_NIN, i = p % MLP_NIN;
      for (int s = 0; s < ns; ++s) g = fmaf(sm.z1[s][o], sm.x[s][i], g);
    } else if (p < MLP_OFF_W2) {
      const int o = p - MLP_OFF_B1;
      for (int s = 0; s < ns; ++s) g += sm.z1[s][o];
    } else if (p < MLP_OFF_B2) {
      const int q = p - MLP_OFF_W2, o = q / MLP_NH, i = q % MLP_NH;
      for (int s = 0; s < ns; ++s) g = fmaf(sm.z2[s][o], sm.h1[s][i], g);
    } else if (p < MLP_OFF_W3) {
      const int o = p - MLP_OFF_B2;
      for (int s = 0; s < ns; ++s) g += sm.z2[s][o];
    } else if (p < MLP_OFF_B3) {
      const int q = p - MLP_OFF_W3, o = q / MLP_NH, i = q % MLP_NH;
      for (int s = 0; s < ns; ++s) g = fmaf(sm.y[s][o], sm.h2[s][i], g);
    } else {
      const int o = p - MLP_OFF_B3;
      for (int s = 0; s < ns; ++s) g += sm.y[s][o];
    }
    out[p] = g;
  }
}

// grad[p] = sum over chunks (in chunk order); loss = sum of loss partials / (nsamp * NOUT)
__global__ void k_mlp_reduce(const float* __restrict__ partial, long long nchunk, float* __restrict__ grad,
                             const float* __restrict__ loss_partial, float* __restrict__ loss, long long nsamp) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < MLP_NPARAM) {
    float g = 0.f;
    for (long long c = 0; c < nchunk; ++c) g += partial[c * MLP_NPARAM + p];
    grad[p] = g;
  }
  if (p == 0 && loss) {
    float t = 0.f;
    for (long long c = 0; c < nchunk; ++c) t += loss_partial[c];
    *loss = t / ((float)nsamp * MLP_NOUT);
  }
}

// AdamW (Loshchilov & Hutter): decoupled weight decay, bias-corrected moments; step >= 1
__global__ void k_adamw(float* __restrict__ params, const float* __restrict__ grad, float* __restrict__ m,
                        float* __restrict__ v, int n, int step, float lr, float b1, float b2, float eps, float wd) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const float g = grad[p];
  const float mm = b1 * m[p] + (1.f - b1) * g;
  const float vv = b2 * v[p] + (1.f - b2) * g * g;
  m[p] = mm;
  v[p] = vv;
  const float mh = mm / (1.f - powf(b1, (float)step));
  const float vh = vv / (1.f - powf(b2, (float)step));
  params[p] -= lr * (mh / (sqrtf(vh) + eps) + wd * params[p]);
}

size_t mlp_smem_bytes() { return sizeof(Smem); }

long long mlp_workspace_floats(long long nsamp) {
  const long long nchunk = (nsamp + S - 1) / S;
  return nchunk * MLP_NPARAM + nchunk;
}

// The shared-memory opt-in of the training kernels is a per-device attribute: set once on every
// device that launches them.
static int set_attr() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return (int)e;
  if (dev < 0 || dev >= 64) return (int)cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev]) return 0;
  e = cudaFuncSetAttribute(k_mlp_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_mlp_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem));
  if (e == cudaSuccess) done[dev] = true;
  return (int)e;
}

int launch_mlp_forward(const float* params, const void* x_bf16, float* y, long long nsamp, void* stream) {
  if (int e = set_attr()) return e;
  const long long nchunk = (nsamp + S - 1) / S;
  const unsigned grid = (unsigned)std::min<long long>(nchunk, 152LL * 2);
  k_mlp_fwd<<<grid, NT, sizeof(Smem), (cudaStream_t)stream>>>(params, (const __nv_bfloat16*)x_bf16, y, nsamp);
  return (int)cudaGetLastError();
}

int launch_mlp_grad(const float* params, const void* x_bf16, const float* target, long long nsamp, float* workspace,
                    float* grad, float* loss, void* stream) {
  if (int e = set_attr()) return e;
  const long long nchunk = (nsamp + S - 1) / S;
  float* partial = workspace;
  float* lpart = workspace + nchunk * MLP_NPARAM;
  cudaStream_t st = (cudaStream_t)stream;
  k_mlp_bwd<<<(unsigned)nchunk, NT, sizeof(Smem), st>>>(params, (const __nv_bfloat16*)x_bf16, target, nsamp, partial, lpart);
  k_mlp_reduce<<<(MLP_NPARAM + 255) / 256, 256, 0, st>>>(partial, nchunk, grad, lpart, loss, nsamp);
  return (int)cudaGetLastError();
}

int launch_adamw(float* params, const float* grad, float* m, float* v, int n, int step, float lr, float b1, float b2,
                 float eps, float wd, void* stream) {
  k_adamw<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, grad, m, v, n, step, lr, b1, b2, eps, wd);
  return (int)cudaGetLastError();
}


// ------------------------------------------------------------------------------- halo columns

namespace {

// Sub-domain-local coordinates of point j (1..HDEPTH) of a face column: the halo point at depth j
// outside face f, or the own point at depth j inside it.  t1, t2 run over the owned extent of the
// two tangential axes (a+1)%3 and (a+2)%3.
__device__ __forceinline__ void column_point(const SubDev& d, int f, int t1, int t2, int j, bool halo, int c[3]) {
  const int a = f >> 1, side = f & 1;
  const int sz[3] = {d.sx, d.sy, d.sz};
  c[(a + 1) % 3] = t1;
  c[(a + 2) % 3] = t2;
  if (halo) c[a] = side == 0 ? -j : sz[a] - 1 + j;
  else c[a] = side == 0 ? j - 1 : sz[a] - j;
}

// index within a state array: the block's offset plus the wrapped point of the block (variable 0);
// column points lie within HDEPTH of the sub-domain, so one conditional wrap per axis suffices
__device__ __forceinline__ long long global_index(const Geometry& g, const SubDev& d, const int c[3]) {
  auto w1 = [](int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); };
  const int gx = w1(d.ox + c[0], d.bnx), gy = w1(d.oy + c[1], d.bny), gz = w1(d.oz + c[2], d.bnz);
  return d.bbase + (long long)gx + (long long)d.bnx * ((long long)gy + (long long)d.bny * gz);
}

// FP64 -> FP32 -> BF16 (FP32 step on the integer pipe: round to nearest, ties away from zero,
// which differs from the FP64 pipe's conversion only on exact FP32 ties)
__device__ __forceinline__ float bf16r(double x) { return __bfloat162float(__float2bfloat16_rn(d2f_fast(x))); }

// Features of depth j of one column: halo level differences (10 values), own-side change (5
// values), the 3-level extrapolation of the halo point (5 values, FP64) and optionally the truth.
// put(e, value) receives feature e of the column.
template <class Put>
__device__ __forceinline__ void column_depth(const Geometry& g, const StepSched& sc, const double* __restrict__ ring,
                                             const SubDev& d, int f, int t1, int t2, int k, int j, const MlpScales& ms,
                                             const double* at3w, Put put, double* at3, double* truth) {
  const long long lvN = 5 * g.N;
  int c[3];
  column_point(d, f, t1, t2, j, true, c);
  const long long gh = global_index(g, d, c);
  column_point(d, f, t1, t2, j, false, c);
  const long long go = global_index(g, d, c);
  // ring slots of levels n, n-k, n-k-1, n-k-2 (k + 2 < R)
  const int nR = (int)(sc.n % sc.R);
  auto slot = [&](int back) { const int q = nR - back; return q < 0 ? q + sc.R : q; };
  const double* Lk0 = ring + (long long)slot(k) * lvN;
  const double* Lk1 = ring + (long long)slot(k + 1) * lvN;
  const double* Lk2 = ring + (long long)slot(k + 2) * lvN;
  const double* Ln = ring + (long long)nR * lvN;
  for (int v = 0; v < 5; ++v) {
    const double a = Lk0[v * d.bN + gh], b = Lk1[v * d.bN + gh], cc = Lk2[v * d.bN + gh];
    put((j - 1) * 5 + v, bf16r((a - b) * ms.in[v]));
    put(MLP_HDEPTH * 5 + (j - 1) * 5 + v, bf16r((b - cc) * ms.in[v]));
    put(2 * MLP_HDEPTH * 5 + (j - 1) * 5 + v, bf16r((Ln[v * d.bN + go] - Lk0[v * d.bN + go]) * ms.own[v]));
    at3[(j - 1) * 5 + v] = fma(at3w[0], a, fma(at3w[1], b, at3w[2] * cc));
    if (truth) truth[(j - 1) * 5 + v] = Ln[v * d.bN + gh];
  }
}

struct At3Table {
  double w[MLP_KMAX + 1][3];
};

}  // namespace

// One thread per training sample spec (sub-domain, face, t1, t2, k).
// at4 (may be null): the residual of the AT4 stage-0 value of Eq. 15 -- the extrapolation from the
// five levels n-k .. n-k-4 with the weights W^(0)(k) = c(k) of the context's table sc.W -- in the
// same units, for comparing the network with the method it would replace.
__global__ void k_halo_samples(Geometry g, StepSched sc, const double* __restrict__ ring, const SubDev* __restrict__ subs,
                               const int* __restrict__ spec, long long n, MlpScales ms, At3Table t3,
                               __nv_bfloat16* __restrict__ x, float* __restrict__ target, float* __restrict__ at4, int s) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int* sp = spec + 5 * i;
  const int sid = sp[0], f = sp[1], t1 = sp[2], t2 = sp[3], k = sp[4];
  const SubDev d = subs[sid];
  float xrow[MLP_NIN];
  double at3[MLP_NOUT], truth[MLP_NOUT];
  auto put = [&](int e, float val) { xrow[e] = val; };
  for (int j = 1; j <= MLP_HDEPTH; ++j) column_depth(g, sc, ring, d, f, t1, t2, k, j, ms, t3.w[k], put, at3, truth);
  for (int q = 0; q <= MLP_KMAX; ++q) xrow[3 * MLP_HDEPTH * 5 + q] = (q == k) ? 1.f : 0.f;
  for (int e = 0; e < MLP_NIN; ++e) x[i * MLP_NIN + e] = __float2bfloat16_rn(xrow[e]);
  for (int e = 0; e < MLP_NOUT; ++e) target[i * MLP_NOUT + e] = (float)((truth[e] - at3[e]) * ms.out[e % 5]);
  if (at4) {
    const long long lvN = 5 * g.N;
    const int nR = (int)(sc.n % sc.R);
    const double* w = sc.W + (long long)k * s * sc.C;  // stage 0: c(k)
    for (int j = 1; j <= MLP_HDEPTH; ++j) {
      int c[3];
      column_point(d, f, t1, t2, j, true, c);
      const long long gh = global_index(g, d, c);
      for (int v = 0; v < 5; ++v) {
        double e = 0.0;
        for (int l = 0; l < sc.C; ++l) {
          const int q = nR - k - l;
          e = fma(w[l], ring[(long long)(q < 0 ? q + sc.R : q) * lvN + v * d.bN + gh], e);
        }
        at4[i * MLP_NOUT + (j - 1) * 5 + v] = (float)((truth[(j - 1) * 5 + v] - e) * ms.out[v]);
      }
    }
  }
}

// Solver use, two launches per asynchronous step.  k_mlp_features: one thread per (face column,
// depth) pair gathers that depth's features at the face's delay (FP64 differences and scaling,
// BF16 rounding) into the column's row of its 128-column tile -- FP32 values in the tensor cores'
// operand layout, so a tile is one contiguous block -- and writes the 3-level extrapolation of the
// halo point to LH (FP64, padded-box layout).  k_mlp_halo: each CTA takes tiles of TM = 128
// columns, fetches a tile's features with one bulk copy (the next tile's copy is issued as soon
// as the first layer has consumed the current one, so it overlaps the rest of the network), runs
// the network on the tensor cores and adds residual / out scale to LH for the HDEPTH halo points
// of each column.
//
// Every layer is one tcgen05 GEMM of M = 128 columns: D[m][n] = sum_k A[m][k] B[n][k] with A (the
// activations) and B (the weights) in shared memory, K-major without swizzle (8-row x 16-byte core
// matrices, K-adjacent cores 128 bytes apart, row groups K/4 x 128 bytes apart), D in tensor
// memory (FP32).  The operands are FP32 values split into TF32 pairs x = hi + lo (hi rounded to 10
// mantissa bits, lo = x - hi exactly); each K step issues hi*hi + hi*lo + lo*hi (kind::tf32, FP32
// accumulation), which keeps the network at FP32 accuracy (the dropped lo*lo and the truncation of
// lo are below 2^-21 relative).  The features are BF16 values, exact in TF32, so the first layer
// needs A_hi only.  One thread issues the MMAs and commits them to an mbarrier; all threads wait
// (bounded), read D with tcgen05.ld (warp w: TMEM lanes 32 (w % 4).., a quarter of the columns),
// add the bias, apply GELU and write the next layer's operands.
namespace {

constexpr int TM = MLP_TILE;  // columns per tile (MMA M)
constexpr int TC_NT = 512;    // threads: 16 warps; warp w reads TMEM lanes 32 (w % 4).. and column quarter w / 4
constexpr int K1 = MLP_K1;    // NIN = 65 padded to a multiple of 8
constexpr unsigned XT_BYTES = TM * K1 * 4;          // one feature tile
constexpr unsigned AT_BYTES = TM * MLP_NOUT * 8;     // one tile's extrapolations
constexpr unsigned FEAT_SMEM = XT_BYTES + AT_BYTES;   // k_mlp_features: one tile of each
constexpr int N3 = 32;        // NOUT = 20 padded to a multiple of 16
constexpr int TMEM_COLS = 256;
constexpr int D1 = 0, D2 = 64, D3 = 128;  // TMEM column of each layer's accumulator
constexpr unsigned MBAR_SPIN_LIMIT = 1u << 22;

struct TcSmem {
  __align__(16) float w1h[MLP_NH * K1];
  __align__(16) float w1l[MLP_NH * K1];
  __align__(16) float w2h[MLP_NH * MLP_NH];
  __align__(16) float w2l[MLP_NH * MLP_NH];
  __align__(16) float w3h[N3 * MLP_NH];
  __align__(16) float w3l[N3 * MLP_NH];
  __align__(16) float x[TM * K1];
  __align__(16) float hh[TM * MLP_NH];
  __align__(16) float hl[TM * MLP_NH];
  float b1[MLP_NH], b2[MLP_NH], b3[N3];
  __align__(16) double at3[TM][MLP_NOUT];  // the tile's 3-level extrapolations
  unsigned long long mbar;
  unsigned long long xbar;  // the bulk copy of a feature tile
  unsigned long long abar;  // the bulk copy of a tile's extrapolations
  unsigned tmem_base;
  int fail;
};

// float index of element (r, k) of an R x K operand in the K-major no-swizzle core layout
__device__ __forceinline__ int core_off(int r, int k, int K) { return ((r >> 3) * (K >> 2) + (k >> 2)) * 32 + (r & 7) * 4 + (k & 3); }

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// TF32 pair: hi = x rounded to 10 mantissa bits, lo = x - hi (exact)
__device__ __forceinline__ void tf32_split(float x, float& hi, float& lo) {
  hi = __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xffffe000u);
  lo = x - hi;
}

// shared-memory matrix descriptor: start, leading (K-direction core) and stride (row-group)
// byte offsets, tcgen05 version 1, no swizzle
__device__ __forceinline__ unsigned long long sdesc(const void* p, unsigned lbo, unsigned sbo) {
  return (unsigned long long)((smem_u32(p) >> 4) & 0x3fffu) | ((unsigned long long)((lbo >> 4) & 0x3fffu) << 16) |
         ((unsigned long long)((sbo >> 4) & 0x3fffu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::tf32: D FP32, A and B TF32, both K-major, N x M = 128
__host__ __device__ constexpr unsigned idesc_tf32(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(n >> 3) << 17) | ((unsigned)(TM >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(unsigned d, unsigned long long a, unsigned long long b, unsigned idesc, int acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(unsigned long long* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ bool mbar_try(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the MMAs committed to the barrier (phase parity); bounded.  Returns false (and every
// thread of the CTA sees the same) when the wait gave up.
__device__ __forceinline__ bool mma_wait(TcSmem& sm, unsigned parity) {
  unsigned it = 0;
  bool ok = true;
  while (!mbar_try(&sm.mbar, parity))
    if (++it > MBAR_SPIN_LIMIT) {
      ok = false;
      break;
    }
  if (!ok) sm.fail = 1;
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  return __syncthreads_and(ok) != 0;
}

// Bounded wait for phase `parity` of a tile-copy barrier; every thread of the CTA sees the same
// result.
__device__ __forceinline__ bool tile_wait(TcSmem& sm, unsigned long long* bar, unsigned parity) {
  unsigned it = 0;
  bool ok = true;
  while (!mbar_try(bar, parity))
    if (++it > MBAR_SPIN_LIMIT) {
      ok = false;
      break;
    }
  if (!ok) sm.fail = 1;
  return __syncthreads_and(ok) != 0;
}

// `bytes` global -> shared by the bulk-copy engine, completing on `bar` (one thread; both
// addresses 16-byte aligned, bytes a multiple of 16).
__device__ __forceinline__ void tile_fetch(unsigned long long* bar, void* dst, const void* src, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(unsigned taddr, float* r) {
  unsigned u[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]), "=r"(u[8]),
        "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) r[i] = __uint_as_float(u[i]);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void async_proxy_fence() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// One layer's MMAs for the tile: K/8 steps of (A_hi B_hi, A_hi B_lo[, A_lo B_hi]).
__device__ __forceinline__ void layer_mma(unsigned d, const float* ah, const float* al, const float* bh, const float* bl,
                                          int K, int N) {
  const unsigned sbo = (unsigned)(K / 4) * 128u, lbo = 128u, id = idesc_tf32(N);
  for (int ks = 0; ks < K / 8; ++ks) {
    const int off = ks * 64;  // 2 cores of 32 floats along K per step
    const unsigned long long a_h = sdesc(ah + off, lbo, sbo), b_h = sdesc(bh + off, lbo, sbo), b_l = sdesc(bl + off, lbo, sbo);
    mma_tf32(d, a_h, b_h, id, ks > 0);
    mma_tf32(d, a_h, b_l, id, 1);
    if (al) mma_tf32(d, sdesc(al + off, lbo, sbo), b_h, id, 1);
  }
}

}  // namespace

// One CTA per tile of TM face columns, one thread per (column, depth): that depth's features
// into the column's row of the tile and the 3-level extrapolation of its halo point, both
// assembled in shared memory (features in the operand layout of the first layer, the depth-1
// thread adding the one-hot delay and the padding; the idle rows of the last tile zero) and
// stored with 16-byte writes: X [tile][TM x K1] FP32, A3 [tile][TM][MLP_NOUT] FP64.
__global__ void __launch_bounds__(TM * MLP_HDEPTH) k_mlp_features(Geometry g, StepSched sc, const double* __restrict__ ring,
                                                                 const SubDev* __restrict__ subs,
                                                                 const int* __restrict__ cols, long long ncol,
                                                                 MlpScales ms, At3Table t3, float* __restrict__ X,
                                                                 double* __restrict__ A3) {
  sc = resolve(sc);
  if (sc.mode != 1) return;  // the network replaces AT halos only
  extern __shared__ __align__(16) unsigned char feat_raw[];
  float* sx = reinterpret_cast<float*>(feat_raw);                         // [TM * K1]
  double* sa = reinterpret_cast<double*>(feat_raw + sizeof(float) * TM * K1);  // [TM * MLP_NOUT]
  const long long tile = blockIdx.x;
  const int tid = threadIdx.x, row = tid >> 2, r = tid & 3;  // depth r + 1
  const long long col = tile * TM + row;
  if (col < ncol) {
    const int* cp = cols + 4 * col;
    const int sid = cp[0], f = cp[1], t1 = cp[2], t2 = cp[3];
    const int k = face_delay(sc, sid, f);
    const SubDev d = subs[sid];
    auto put = [&](int q, float val) { sx[core_off(row, q, K1)] = val; };
    column_depth(g, sc, ring, d, f, t1, t2, k, r + 1, ms, t3.w[k], put, sa + row * MLP_NOUT, nullptr);
    if (r == 0)
      for (int q = 3 * MLP_HDEPTH * 5; q < K1; ++q) put(q, (q - 3 * MLP_HDEPTH * 5 == k) ? 1.f : 0.f);  // one-hot, padding
  } else {
    for (int q = r; q < K1; q += 4) sx[core_off(row, q, K1)] = 0.f;
#pragma unroll
    for (int v = 0; v < 5; ++v) sa[row * MLP_NOUT + 5 * r + v] = 0.0;
  }
  __syncthreads();
  float4* gx = reinterpret_cast<float4*>(X + tile * (TM * K1));
  const float4* s4 = reinterpret_cast<const float4*>(sx);
  for (int i = tid; i < TM * K1 / 4; i += TM * MLP_HDEPTH) gx[i] = s4[i];
  double2* ga = reinterpret_cast<double2*>(A3 + tile * (TM * MLP_NOUT));
  const double2* s2 = reinterpret_cast<const double2*>(sa);
  for (int i = tid; i < TM * MLP_NOUT / 2; i += TM * MLP_HDEPTH) ga[i] = s2[i];
}

__global__ void __launch_bounds__(TC_NT, 1) k_mlp_halo(Geometry g, StepSched sc, const SubDev* __restrict__ subs,
                                                        const int* __restrict__ cols, long long ncol,
                                                        const float* __restrict__ params, MlpScales ms,
                                                        const float* __restrict__ X, const double* __restrict__ A3,
                                                        double* __restrict__ LH) {
  sc = resolve(sc);
  if (sc.mode != 1) return;  // the network replaces AT halos only
  extern __shared__ __align__(16) unsigned char tc_raw[];
  TcSmem& sm = *reinterpret_cast<TcSmem*>(tc_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // tensor memory (one warp allocates; the whole CTA frees it at the end) and the barrier
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&sm.tmem_base)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&sm.mbar)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&sm.xbar)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&sm.abar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    sm.fail = 0;
  }
  // weights as TF32 pairs in the core layout (padding zero), biases
  for (int p = tid; p < MLP_NH * K1; p += TC_NT) {
    const int n = p / K1, k = p % K1;
    float h = 0.f, l = 0.f;
    if (k < MLP_NIN) tf32_split(params[MLP_OFF_W1 + n * MLP_NIN + k], h, l);
    sm.w1h[core_off(n, k, K1)] = h;
    sm.w1l[core_off(n, k, K1)] = l;
  }
  for (int p = tid; p < MLP_NH * MLP_NH; p += TC_NT) {
    const int n = p / MLP_NH, k = p % MLP_NH;
    float h, l;
    tf32_split(params[MLP_OFF_W2 + p], h, l);
    sm.w2h[core_off(n, k, MLP_NH)] = h;
    sm.w2l[core_off(n, k, MLP_NH)] = l;
  }
  for (int p = tid; p < N3 * MLP_NH; p += TC_NT) {
    const int n = p / MLP_NH, k = p % MLP_NH;
    float h = 0.f, l = 0.f;
    if (n < MLP_NOUT) tf32_split(params[MLP_OFF_W3 + p], h, l);
    sm.w3h[core_off(n, k, MLP_NH)] = h;
    sm.w3l[core_off(n, k, MLP_NH)] = l;
  }
  for (int p = tid; p < MLP_NH; p += TC_NT) {
    sm.b1[p] = params[MLP_OFF_B1 + p];
    sm.b2[p] = params[MLP_OFF_B2 + p];
  }
  for (int p = tid; p < N3; p += TC_NT) sm.b3[p] = p < MLP_NOUT ? params[MLP_OFF_B3 + p] : 0.f;
  double inv_out[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) inv_out[v] = 1.0 / ms.out[v];
  tc_fence_before();
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const unsigned tmem = sm.tmem_base;
  // this warp's TMEM lanes (rows 32 q..) and column quarter
  const int q = warp & 3, quarter = warp >> 2, row = 32 * q + lane;
  const unsigned lane_addr = tmem + ((unsigned)(32 * q) << 16);
  unsigned parity = 0, xparity = 0, aparity = 0;
  bool ok = true;
  // the first tile's features and extrapolations (the barriers were initialised before the
  // block-wide barrier above)
  if (tid == 0 && (long long)blockIdx.x * TM < ncol) {
    tile_fetch(&sm.xbar, sm.x, X + (long long)blockIdx.x * (TM * K1), XT_BYTES);
    tile_fetch(&sm.abar, sm.at3, A3 + (long long)blockIdx.x * (TM * MLP_NOUT), AT_BYTES);
  }

  for (long long base = (long long)blockIdx.x * TM; ok && base < ncol; base += (long long)gridDim.x * TM) {
    const int ns = (int)min((long long)TM, ncol - base);
    const long long tile = base / TM, ntile_next = tile + gridDim.x;
    if (!(ok = tile_wait(sm, &sm.xbar, xparity))) break;
    xparity ^= 1;
    // ---- layer 1: z1 = x W1^T (+ b1 below)
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      layer_mma(tmem + D1, sm.x, nullptr, sm.w1h, sm.w1l, K1, MLP_NH);
      mma_commit(&sm.mbar);
    }
    if (!(ok = mma_wait(sm, parity))) break;
    parity ^= 1;
    // the first layer has read this tile's features: fetch the next tile's during the rest
    if (tid == 0 && ntile_next * TM < ncol) tile_fetch(&sm.xbar, sm.x, X + ntile_next * (TM * K1), XT_BYTES);
    // ---- epilogue: h = GELU(z + b) as TF32 pairs; warp reads 16 of the 64 columns of its rows
    auto hidden = [&](int dcol, const float* b) {
      float z[16];
      tmem_ld16(lane_addr + (unsigned)(dcol + 16 * quarter), z);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int n = 16 * quarter + i;
        float h, l;
        tf32_split(gelu(z[i] + b[n]), h, l);
        sm.hh[core_off(row, n, MLP_NH)] = h;
        sm.hl[core_off(row, n, MLP_NH)] = l;
      }
      async_proxy_fence();
      tc_fence_before();
      __syncthreads();
    };
    hidden(D1, sm.b1);
    // ---- layer 2
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      layer_mma(tmem + D2, sm.hh, sm.hl, sm.w2h, sm.w2l, MLP_NH, MLP_NH);
      mma_commit(&sm.mbar);
    }
    if (!(ok = mma_wait(sm, parity))) break;
    parity ^= 1;
    hidden(D2, sm.b2);
    // ---- layer 3
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      layer_mma(tmem + D3, sm.hh, sm.hl, sm.w3h, sm.w3l, MLP_NH, N3);
      mma_commit(&sm.mbar);
    }
    if (!(ok = mma_wait(sm, parity))) break;
    parity ^= 1;
    // ---- outputs: warp quarter c holds outputs 8c..8c+7 of its rows (20 of the 32 used)
    if (!(ok = tile_wait(sm, &sm.abar, aparity))) break;
    aparity ^= 1;
    {
      float y[8];
      unsigned u[8];
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                   : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7])
                   : "r"(lane_addr + (unsigned)(D3 + 8 * quarter)));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
      for (int i = 0; i < 8; ++i) y[i] = __uint_as_float(u[i]);
      if (row < ns && 8 * quarter < MLP_NOUT) {
        const int* cp = cols + 4 * (base + row);
        const SubDev d = subs[cp[0]];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int o = 8 * quarter + i;
          if (o >= MLP_NOUT) continue;
          const int j = o / 5 + 1, v = o % 5;
          int c[3];
          column_point(d, cp[1], cp[2], cp[3], j, true, c);
          const long long qq =
              (long long)(c[0] + g.G) + (long long)d.ex * ((long long)(c[1] + g.G) + (long long)d.ey * (c[2] + g.Gz));
          double iv = inv_out[0];
#pragma unroll
          for (int vv = 1; vv < 5; ++vv) iv = v == vv ? inv_out[vv] : iv;
          LH[(long long)v * g.Ptot + d.pbase + qq] = fma((double)(y[i] + sm.b3[o]), iv, sm.at3[row][o]);
        }
      }
    }
    tc_fence_before();
    __syncthreads();
    // this tile's extrapolations are read (generic loads, ordered before the async-proxy copy
    // that overwrites them by the barrier and the proxy fence): fetch the next tile's
    if (tid == 0 && ntile_next * TM < ncol) {
      async_proxy_fence();
      tile_fetch(&sm.abar, sm.at3, A3 + ntile_next * (TM * MLP_NOUT), AT_BYTES);
    }
  }
  // a wait that gave up: record it in the status word (the host reports CFS_ETIMEOUT) and poison
  // this CTA's columns so the state shows it too
  if (!ok) {
    if (tid == 0 && sc.status) atomicOr(sc.status, 1);
    for (long long base = (long long)blockIdx.x * TM; base < ncol; base += (long long)gridDim.x * TM)
      for (int e = tid; e < TM * MLP_NOUT && base + e / MLP_NOUT < ncol; e += TC_NT) {
        const int col = e / MLP_NOUT, o = e % MLP_NOUT, j = o / 5 + 1, v = o % 5;
        const int* cp = cols + 4 * (base + col);
        const SubDev d = subs[cp[0]];
        int c[3];
        column_point(d, cp[1], cp[2], cp[3], j, true, c);
        const long long qq =
            (long long)(c[0] + g.G) + (long long)d.ex * ((long long)(c[1] + g.G) + (long long)d.ey * (c[2] + g.Gz));
        LH[(long long)v * g.Ptot + d.pbase + qq] = __longlong_as_double(0x7ff8000000000000LL);
      }
    // give MMAs and a feature copy still in flight a bounded chance to finish before the memory
    // they use is freed
    for (unsigned it = 0; it < MBAR_SPIN_LIMIT && !mbar_try(&sm.mbar, parity); ++it) {
    }
    for (unsigned it = 0; it < MBAR_SPIN_LIMIT && !mbar_try(&sm.xbar, xparity); ++it) {
    }
    for (unsigned it = 0; it < MBAR_SPIN_LIMIT && !mbar_try(&sm.abar, aparity); ++it) {
    }
    __syncthreads();
  }
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

static At3Table at3_table() {
  At3Table t{};
  for (int k = 0; k <= MLP_KMAX; ++k) {
    long double c[5];
    extrap_weights(2, k, c);  // the three-level (second-order) extrapolation of Eq. 14
    for (int l = 0; l < 3; ++l) t.w[k][l] = (double)c[l];
  }
  return t;
}

int launch_halo_samples(const Geometry& g, const StepSched& sc, const double* ring, const SubDev* subs, const int* spec,
                        long long n, MlpScales ms, void* x_bf16, float* target, float* at4, int s, void* stream) {
  if (n <= 0) return 0;
  k_halo_samples<<<(unsigned)((n + 127) / 128), 128, 0, (cudaStream_t)stream>>>(
      g, sc, ring, subs, spec, n, ms, at3_table(), (__nv_bfloat16*)x_bf16, target, at4, s);
  return (int)cudaGetLastError();
}

int launch_mlp_halo(const Geometry& g, const StepSched& sc, const double* ring, const SubDev* subs, const int* cols,
                    long long ncol, const float* params, MlpScales ms, float* X, double* A3, double* LH,
                    void* stream, long long* launches, const Timer* tm) {
  // the shared-memory opt-in is a per-device attribute: set once on every device that launches
  static std::mutex mu;
  static bool attr[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return (int)e;
  if (dev < 0 || dev >= 64) return (int)cudaErrorInvalidDevice;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!attr[dev]) {
      e = cudaFuncSetAttribute(k_mlp_halo, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TcSmem));
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_mlp_features, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FEAT_SMEM);
      if (e != cudaSuccess) return (int)e;
      attr[dev] = true;
    }
  }
  const long long ntile = (ncol + TM - 1) / TM;
  const unsigned grid = (unsigned)std::min<long long>(ntile, 152LL);
  const cudaStream_t st = (cudaStream_t)stream;
  if (tm) tm->rec(tm->self, 0, 1);
  k_mlp_features<<<(unsigned)ntile, TM * MLP_HDEPTH, FEAT_SMEM, st>>>(g, sc, ring, subs, cols, ncol, ms, at3_table(), X, A3);
  k_mlp_halo<<<grid, TC_NT, sizeof(TcSmem), st>>>(g, sc, subs, cols, ncol, params, ms, X, A3, LH);
  if (tm) tm->rec(tm->self, 0, 0);
  if (launches) *launches += 2;
  return (int)cudaGetLastError();
}

}  // namespace cfs
