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

static bool g_attr = false;

static int set_attr() {
  if (g_attr) return 0;
  cudaError_t e = cudaFuncSetAttribute(k_mlp_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_mlp_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem));
  if (e == cudaSuccess) g_attr = true;
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
// Feature e of the column goes to xrow[e * xs].
__device__ __forceinline__ void column_depth(const Geometry& g, const StepSched& sc, const double* __restrict__ ring,
                                             const SubDev& d, int f, int t1, int t2, int k, int j, const MlpScales& ms,
                                             const double* at3w, float* xrow, int xs, double* at3, double* truth) {
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
    xrow[((j - 1) * 5 + v) * xs] = bf16r((a - b) * ms.in[v]);
    xrow[(MLP_HDEPTH * 5 + (j - 1) * 5 + v) * xs] = bf16r((b - cc) * ms.in[v]);
    xrow[(2 * MLP_HDEPTH * 5 + (j - 1) * 5 + v) * xs] = bf16r((Ln[v * d.bN + go] - Lk0[v * d.bN + go]) * ms.own[v]);
    at3[(j - 1) * 5 + v] = fma(at3w[0], a, fma(at3w[1], b, at3w[2] * cc));
    if (truth) truth[(j - 1) * 5 + v] = Ln[v * d.bN + gh];
  }
}

struct At3Table {
  double w[MLP_KMAX + 1][3];
};

}  // namespace

// One thread per training sample spec (sub-domain, face, t1, t2, k).
__global__ void k_halo_samples(Geometry g, StepSched sc, const double* __restrict__ ring, const SubDev* __restrict__ subs,
                               const int* __restrict__ spec, long long n, MlpScales ms, At3Table t3,
                               __nv_bfloat16* __restrict__ x, float* __restrict__ target) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int* sp = spec + 5 * i;
  const int sid = sp[0], f = sp[1], t1 = sp[2], t2 = sp[3], k = sp[4];
  const SubDev d = subs[sid];
  float xrow[MLP_NIN];
  double at3[MLP_NOUT], truth[MLP_NOUT];
  for (int j = 1; j <= MLP_HDEPTH; ++j) column_depth(g, sc, ring, d, f, t1, t2, k, j, ms, t3.w[k], xrow, 1, at3, truth);
  for (int q = 0; q <= MLP_KMAX; ++q) xrow[3 * MLP_HDEPTH * 5 + q] = (q == k) ? 1.f : 0.f;
  for (int e = 0; e < MLP_NIN; ++e) x[i * MLP_NIN + e] = __float2bfloat16_rn(xrow[e]);
  for (int e = 0; e < MLP_NOUT; ++e) target[i * MLP_NOUT + e] = (float)((truth[e] - at3[e]) * ms.out[e % 5]);
}

// Solver use: each CTA takes SP face columns (sub-domain, face, t1, t2) at a time, gathers their
// features at the face's delay (one thread per column depth), runs the network and writes
// U^(0) = extrapolation + residual / out scale for the HDEPTH halo points of each column into LH
// (FP64, padded-box layout).  The layers are register-blocked: a thread computes 4 samples x 4
// outputs from float4 loads of the transposed activations and weights (two shared-memory loads
// per 16 FMA); every output accumulates its inputs in the same order as the training kernels,
// so inference gives the same bits.
namespace {

constexpr int SP = 64;                       // columns per CTA iteration
constexpr int NOUTP = 20;                    // NOUT, a multiple of 4

struct HaloSmem {
  __align__(16) float wT1[MLP_NIN][MLP_NH];
  __align__(16) float b1[MLP_NH];
  __align__(16) float wT2[MLP_NH][MLP_NH];
  __align__(16) float b2[MLP_NH];
  __align__(16) float wT3[MLP_NH][NOUTP];
  __align__(16) float b3[NOUTP];
  __align__(16) float xT[MLP_NIN][SP];
  __align__(16) float h1T[MLP_NH][SP];
  __align__(16) float h2T[MLP_NH][SP];
  __align__(16) float yT[NOUTP][SP];
  double at3[SP][MLP_NOUT];
};

// out^T[o][s] = act(b[o] + sum_i W[o][i] in[s][i]) with transposed operands wT[i][o], inT[i][s].
template <int NIN, int NOUT, bool ACT>
__device__ __forceinline__ void layer_blocked(const float (*wT)[NOUT], const float* b, const float (*inT)[SP],
                                              float (*outT)[SP]) {
  constexpr int NOG = NOUT / 4, NSG = SP / 4;
  for (int t = threadIdx.x; t < NOG * NSG; t += NT) {
    const int og = t % NOG, sg = t / NOG;
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][c] = b[4 * og + c];
#pragma unroll 5
    for (int i = 0; i < NIN; ++i) {
      const float4 xv = *reinterpret_cast<const float4*>(&inT[i][4 * sg]);
      const float4 wv = *reinterpret_cast<const float4*>(&wT[i][4 * og]);
      const float xa[4] = {xv.x, xv.y, xv.z, xv.w}, wc[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = fmaf(wc[c], xa[a], acc[a][c]);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int a = 0; a < 4; ++a) outT[4 * og + c][4 * sg + a] = ACT ? gelu(acc[a][c]) : acc[a][c];
  }
}

}  // namespace

__global__ void __launch_bounds__(NT, 2) k_mlp_halo(Geometry g, StepSched sc, const double* __restrict__ ring,
                                                     const SubDev* __restrict__ subs, const int* __restrict__ cols,
                                                     long long ncol, const float* __restrict__ params, MlpScales ms,
                                                     At3Table t3, double* __restrict__ LH) {
  sc = resolve(sc);
  if (sc.mode != 1) return;  // the network replaces AT halos only
  extern __shared__ __align__(16) unsigned char raw[];
  HaloSmem& sm = *reinterpret_cast<HaloSmem*>(raw);
  // reciprocal output scales (one division per thread instead of one per output)
  double inv_out[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) inv_out[v] = 1.0 / ms.out[v];
  // weights transposed once per CTA
  for (int p = threadIdx.x; p < MLP_NH * MLP_NIN; p += NT) sm.wT1[p % MLP_NIN][p / MLP_NIN] = params[MLP_OFF_W1 + p];
  for (int p = threadIdx.x; p < MLP_NH * MLP_NH; p += NT) sm.wT2[p % MLP_NH][p / MLP_NH] = params[MLP_OFF_W2 + p];
  for (int p = threadIdx.x; p < MLP_NOUT * MLP_NH; p += NT) sm.wT3[p % MLP_NH][p / MLP_NH] = params[MLP_OFF_W3 + p];
  for (int p = threadIdx.x; p < MLP_NH; p += NT) {
    sm.b1[p] = params[MLP_OFF_B1 + p];
    sm.b2[p] = params[MLP_OFF_B2 + p];
  }
  for (int p = threadIdx.x; p < NOUTP; p += NT) sm.b3[p] = params[MLP_OFF_B3 + p];
  for (long long base = (long long)blockIdx.x * SP; base < ncol; base += (long long)gridDim.x * SP) {
    const int ns = (int)min((long long)SP, ncol - base);
    // gather: 4 threads per column, thread r handles depth r + 1 (features are per depth)
    {
      const int col = threadIdx.x / MLP_HDEPTH, r = threadIdx.x % MLP_HDEPTH;
      if (col < ns) {
        const int* cp = cols + 4 * (base + col);
        const int sid = cp[0], f = cp[1], t1 = cp[2], t2 = cp[3];
        const int k = face_delay(sc, sid, f);
        column_depth(g, sc, ring, subs[sid], f, t1, t2, k, r + 1, ms, t3.w[k], &sm.xT[0][col], SP, sm.at3[col], nullptr);
        if (r == 0)
          for (int q = 0; q <= MLP_KMAX; ++q) sm.xT[3 * MLP_HDEPTH * 5 + q][col] = (q == k) ? 1.f : 0.f;
      } else if (col < SP && r == 0) {
        for (int i = 0; i < MLP_NIN; ++i) sm.xT[i][col] = 0.f;  // idle columns of a partial chunk
      }
    }
    __syncthreads();
    layer_blocked<MLP_NIN, MLP_NH, true>(sm.wT1, sm.b1, sm.xT, sm.h1T);
    __syncthreads();
    layer_blocked<MLP_NH, MLP_NH, true>(sm.wT2, sm.b2, sm.h1T, sm.h2T);
    __syncthreads();
    layer_blocked<MLP_NH, NOUTP, false>(sm.wT3, sm.b3, sm.h2T, sm.yT);
    __syncthreads();
    for (int e = threadIdx.x; e < ns * MLP_NOUT; e += NT) {
      const int col = e / MLP_NOUT, o = e % MLP_NOUT, j = o / 5 + 1, v = o % 5;
      const int* cp = cols + 4 * (base + col);
      const SubDev d = subs[cp[0]];
      int c[3];
      column_point(d, cp[1], cp[2], cp[3], j, true, c);
      const long long q = (long long)(c[0] + g.G) + (long long)d.ex * ((long long)(c[1] + g.G) + (long long)d.ey * (c[2] + g.Gz));
      double iv = inv_out[0];
#pragma unroll
      for (int vv = 1; vv < 5; ++vv) iv = v == vv ? inv_out[vv] : iv;
      LH[(long long)v * g.Ptot + d.pbase + q] = fma((double)sm.yT[o][col], iv, sm.at3[col][o]);
    }
    __syncthreads();
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
                        long long n, MlpScales ms, void* x_bf16, float* target, void* stream) {
  if (n <= 0) return 0;
  k_halo_samples<<<(unsigned)((n + 127) / 128), 128, 0, (cudaStream_t)stream>>>(
      g, sc, ring, subs, spec, n, ms, at3_table(), (__nv_bfloat16*)x_bf16, target);
  return (int)cudaGetLastError();
}

int launch_mlp_halo(const Geometry& g, const StepSched& sc, const double* ring, const SubDev* subs, const int* cols,
                    long long ncol, const float* params, MlpScales ms, double* LH, void* stream, long long* launches,
                    const Timer* tm) {
  if (int e = set_attr()) return e;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_mlp_halo, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(HaloSmem));
    if (e != cudaSuccess) return (int)e;
    attr = true;
  }
  const long long nchunk = (ncol + SP - 1) / SP;
  const unsigned grid = (unsigned)std::min<long long>(nchunk, 152LL * 2);
  if (tm) tm->rec(tm->self, 0, 1);
  k_mlp_halo<<<grid, NT, sizeof(HaloSmem), (cudaStream_t)stream>>>(g, sc, ring, subs, cols, ncol, params, ms, at3_table(), LH);
  if (tm) tm->rec(tm->self, 0, 0);
  if (launches) *launches += 1;
  return (int)cudaGetLastError();
}

}  // namespace cfs
