// fused.cu -- fused LSERK stage for the FP32-intermediate form (3-D Navier-Stokes, CD4/AT4).
//
// One launch per RK stage (Eq. 3) does what k_view + k_flux + k_rk do in three: each CTA owns an
// FX x FY column tile of one sub-domain and marches through its z-planes, keeping a ring of five
// planes of FP32 primitives (tile + halo of 4) in shared memory:
//   load plane L        own points and synchronous halos from the FP64 stage input; AT/AS halo
//                       points from the per-step halo store (k_halo_prims);
//   plane G = L - 2     CD4 gradients (x, y from the plane, z from the ring), viscous stresses and
//                       heat flux (Eq. A3-A4), combined fluxes Phi_a = -F_a + Fv_a/Re (Eq. A2):
//                       Phi_x, Phi_y of the tile and its x / y strips to shared memory, Phi_z of
//                       the tile to a register queue; then dt (D_x Phi_x + D_y Phi_y) of the tile;
//   plane z = L - 4     dt R = that in-plane part + dt D_z Phi_z from the queue, and the FP64
//                       low-storage update Q = A Q + dt R, U^(m) = U^(m-1) + B Q.
// k_halo_prims runs once per asynchronous step: for every halo point a sub-domain reads from a
// neighbour it applies the AT weights of all s stages to the C delayed levels in FP64 (Eq. 14-15
// and the buffer updates of Eq. 8 / Table 5) and stores the FP32 primitives per stage.
#include <cuda_runtime.h>

#include "cfs_internal.h"
#include "device_common.cuh"

namespace cfs {

namespace {

constexpr int HB = 4;  // halo of the box: 2r for the viscous CD4 operator

// FP32 primitives from an FP64 conserved state; p and rho E are carried as deviations from the
// reference state (p_ref = 1/(gamma M^2), E_ref = p_ref/(gamma-1)).
__device__ __forceinline__ void prims32(const double* u, const Physics& ph, float* w) {
  const float rho = (float)u[0];
  const float ir = 1.0f / rho;
  const float uu = (float)u[1] * ir, vv = (float)u[2] * ir, ww = (float)u[3] * ir;
  const float ke = 0.5f * ((float)u[1] * uu + (float)u[2] * vv + (float)u[3] * ww);
  const float rE = (float)(u[4] - ph.E_ref);
  const float p = (float)ph.gm1 * (rE - ke);
  w[0] = rho;
  w[1] = uu;
  w[2] = vv;
  w[3] = ww;
  w[4] = p;
  w[5] = ((float)ph.gM2 * p + 1.0f) * ir;  // T
  w[6] = rE + p;                          // rho E + p - H_ref
}

}  // namespace

// ------------------------------------------------------------------------------- k_halo_prims

__global__ void __launch_bounds__(256) k_halo_prims(Geometry g, Physics ph, StepSched sc, const double* __restrict__ ring,
                                                    const SubDev* __restrict__ subs, const int2* __restrict__ halo,
                                                    long long nhalo, float* __restrict__ Wh, int s) {
  sc = resolve(sc);
  if (sc.mode == 0) return;  // synchronous step: no halo store is read
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nhalo) return;
  const int2 hv = halo[e];
  const int sid = hv.x;
  const long long t = hv.y;
  const SubDev d = subs[sid];
  const int i = (int)(t % d.ex), j = (int)((t / d.ex) % d.ey), k = (int)(t / ((long long)d.ex * d.ey));
  const int ci = i - g.G, cj = j - g.G, ck = k - g.Gz;
  int kd = 0;
  if (ci < 0 || ci >= d.sx) kd = max(kd, face_delay(sc, sid, ci < 0 ? 0 : 1));
  if (cj < 0 || cj >= d.sy) kd = max(kd, face_delay(sc, sid, cj < 0 ? 2 : 3));
  if (ck < 0 || ck >= d.sz) kd = max(kd, face_delay(sc, sid, ck < 0 ? 4 : 5));
  const int gx = wrapc(d.ox + ci, d.bnx), gy = wrapc(d.oy + cj, d.bny), gz = wrapc(d.oz + ck, d.bnz);
  const long long gi = d.bbase + (long long)gx + (long long)d.bnx * ((long long)gy + (long long)d.bny * gz);
  const long long lvN = 5 * g.N, P = g.Ptot, o = d.pbase + t;
  if (sc.mode == 2) {  // AS: the latest visible level, the same for every stage
    const double* src = ring + (long long)((sc.n - kd) % sc.R) * lvN;
    double u[5];
    for (int v = 0; v < 5; ++v) u[v] = src[v * d.bN + gi];
    float w[7];
    prims32(u, ph, w);
    for (int c = 0; c < 7; ++c) Wh[(long long)c * P + o] = w[c];
    return;
  }
  // AT: U_buf^(m) = sum_l W^(m)_l(k) U^{n-k-l} for every stage m, accumulated in FP64; with the
  // learned halo, face points start from the network's stage-0 value and add (W^(m) - W^(0)) R
  const bool learned = sc.LH && ((int)(ci < 0 || ci >= d.sx) + (int)(cj < 0 || cj >= d.sy) + (int)(ck < 0 || ck >= d.sz) == 1);
  double acc[CFS_MAX_STAGES][5];
  for (int m = 0; m < s; ++m)
    for (int v = 0; v < 5; ++v) acc[m][v] = learned ? sc.LH[(long long)v * g.Ptot + d.pbase + t] : 0.0;
  for (int l = 0; l < sc.C; ++l) {
    const double* src = ring + (long long)((sc.n - kd - l) % sc.R) * lvN;
    double r[5];
    for (int v = 0; v < 5; ++v) r[v] = src[v * d.bN + gi];
    const double w0 = learned ? __ldg(sc.W + (kd * s) * sc.C + l) : 0.0;
    for (int m = learned ? 1 : 0; m < s; ++m) {
      const double wl = __ldg(sc.W + (kd * s + m) * sc.C + l) - w0;
      for (int v = 0; v < 5; ++v) acc[m][v] = fma(wl, r[v], acc[m][v]);
    }
  }
  for (int m = 0; m < s; ++m) {
    float w[7];
    prims32(acc[m], ph, w);
    for (int c = 0; c < 7; ++c) Wh[(long long)(m * 7 + c) * P + o] = w[c];
  }
}

// ------------------------------------------------------------------------------- k_stage_fused

template <int FX, int FY>
struct FusedSmem {
  static constexpr int BX = FX + 2 * HB, BY = FY + 2 * HB;
  static constexpr int W = 5 * 7 * BY * BX;      // ring of 5 planes of 7 primitives
  static constexpr int FXS = 5 * FY * (FX + 4);  // Phi_x of tile + x strips
  static constexpr int FYS = 5 * (FY + 4) * FX;  // Phi_y of tile + y strips
  static constexpr size_t bytes = sizeof(float) * (W + FXS + FYS);
};

template <int FX, int FY>
__global__ void __launch_bounds__(FX* FY) k_stage_fused(Geometry g, Physics ph, StepSched sc,
                                                        const double* __restrict__ Uin0, double* __restrict__ Uout0,
                                                        const double* __restrict__ ring, int in_ring, int out_ring,
                                                        double* __restrict__ Q, const SubDev* __restrict__ subs,
                                                        const int* __restrict__ work, int nwork,
                                                        const float* __restrict__ Wh, int stage, double A, double B,
                                                        double dt, int first, int last) {
  sc = resolve(sc);
  const double* __restrict__ Uin = ring_or(Uin0, in_ring, ring, sc, 0);
  double* __restrict__ Uout = const_cast<double*>(ring_or(Uout0, out_ring, ring, sc, 1));
  using S = FusedSmem<FX, FY>;
  constexpr int BX = S::BX, BY = S::BY, NT = FX * FY, PL = 7 * BY * BX;
  extern __shared__ float smem[];
  float* sW = smem;
  float* sFx = smem + S::W;
  float* sFy = sFx + S::FXS;
  const int tid = threadIdx.x, tx = tid % FX, ty = tid / FX;
  const float ire = (float)ph.ire, kap = (float)ph.kappa, Href = (float)ph.H_ref;
  const int hslot = (sc.mode == 2) ? 0 : stage;

  for (int wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
    const int* wk = work + 4 * wi;  // (sub-domain, x0, y0, z0 | z1 << 16)
    const SubDev d = subs[wk[0]];
    const int tx0 = wk[1], ty0 = wk[2];
    const int z0 = wk[3] & 0xffff, z1 = wk[3] >> 16;  // output planes [z0, z1) of the sub-domain
    const float c1x = (float)d.c1[0], c2x = (float)d.c2[0], c1y = (float)d.c1[1], c2y = (float)d.c2[1];
    const float c1z = (float)d.c1[2], c2z = (float)d.c2[2];
    const float k1x = (float)(dt * d.c1[0]), k2x = (float)(dt * d.c2[0]);
    const float k1y = (float)(dt * d.c1[1]), k2y = (float)(dt * d.c2[1]);
    const float k1z = (float)(dt * d.c1[2]), k2z = (float)(dt * d.c2[2]);
    float phiz[5][5], rxy[3][5];
#pragma unroll
    for (int a = 0; a < 5; ++a)
#pragma unroll
      for (int c = 0; c < 5; ++c) phiz[a][c] = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int c = 0; c < 5; ++c) rxy[a][c] = 0.f;

    for (int L = z0 - HB; L < z1 + HB; ++L) {
      // ---- load plane L (sub-domain local z) into ring slot
      {
        float* dst = sW + ((L + 10) % 5) * PL;
        const int lz = L;
        const int dz = lz < 0 ? -lz : (lz >= d.sz ? lz - d.sz + 1 : 0);
        for (int p = tid; p < BX * BY; p += NT) {
          const int i = p % BX, j = p / BX;
          const int lx = tx0 - HB + i, ly = ty0 - HB + j;
          const int dx = lx < 0 ? -lx : (lx >= d.sx ? lx - d.sx + 1 : 0);
          const int dy = ly < 0 ? -ly : (ly >= d.sy ? ly - d.sy + 1 : 0);
          const int nout = (dx > 0) + (dy > 0) + (dz > 0);
          // the sub-domain's view: faces up to depth HB, edges up to r x r (a narrow ragged tile's
          // box reaches further; those points feed no output and read the stage input instead)
          const bool inview = (nout == 1 && dx <= HB && dy <= HB && dz <= HB) ||
                              (nout == 2 && dx <= g.r && dy <= g.r && dz <= g.r);
          float w[7];
          if (nout == 0 || sc.mode == 0 || !inview) {
            // own point, synchronous halo, or a box point no output depends on: the stage input
            const int gx = wrapc(d.ox + lx, d.bnx), gy = wrapc(d.oy + ly, d.bny), gz = wrapc(d.oz + lz, d.bnz);
            const long long gi = d.bbase + (long long)gx + (long long)d.bnx * ((long long)gy + (long long)d.bny * gz);
            double u[5];
#pragma unroll
            for (int v = 0; v < 5; ++v) u[v] = Uin[v * d.bN + gi];
            prims32(u, ph, w);
          } else {
            const long long q = (long long)(lx + g.G) + (long long)d.ex * ((long long)(ly + g.G) + (long long)d.ey * (lz + g.Gz));
            const float* src = Wh + (long long)hslot * 7 * g.Ptot + d.pbase + q;
#pragma unroll
            for (int c = 0; c < 7; ++c) w[c] = src[(long long)c * g.Ptot];
          }
#pragma unroll
          for (int c = 0; c < 7; ++c) dst[c * BY * BX + j * BX + i] = w[c];
        }
      }
      __syncthreads();
      const int G = L - 2;
      if (G >= z0 - 2 && G <= z1 + 1) {
        const float* pl[5];
#pragma unroll
        for (int o = 0; o < 5; ++o) pl[o] = sW + ((G - 2 + o + 10) % 5) * PL;  // planes G-2..G+2
        const bool strips = (G >= z0 && G < z1);
        float fz[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        // one gradient/flux evaluation at box point (bi, bj) of plane G: kind 0 tile point
        // (Phi_x, Phi_y to shared memory, Phi_z to the queue), 1 x-strip (Phi_x), 2 y-strip (Phi_y)
        auto point = [&](int bi, int bj, int kind) {
          const float* P0 = pl[2];
          const int q = bj * BX + bi;
          auto at = [&](const float* plane, int c, int qq) { return plane[c * BY * BX + qq]; };
          // gradients of u, v, w, T
          float du[3][3], dT[3];
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            const int c = v == 3 ? 5 : 1 + v;
            const float gx_ = c1x * (at(P0, c, q + 1) - at(P0, c, q - 1)) + c2x * (at(P0, c, q + 2) - at(P0, c, q - 2));
            const float gy_ = c1y * (at(P0, c, q + BX) - at(P0, c, q - BX)) + c2y * (at(P0, c, q + 2 * BX) - at(P0, c, q - 2 * BX));
            const float gz_ = c1z * (at(pl[3], c, q) - at(pl[1], c, q)) + c2z * (at(pl[4], c, q) - at(pl[0], c, q));
            if (v < 3) { du[v][0] = gx_; du[v][1] = gy_; du[v][2] = gz_; }
            else { dT[0] = gx_; dT[1] = gy_; dT[2] = gz_; }
          }
          const float rho = at(P0, 0, q), u = at(P0, 1, q), v = at(P0, 2, q), w = at(P0, 3, q);
          const float p = at(P0, 4, q), T = at(P0, 5, q), et = at(P0, 6, q);
          float mu = 1.f;
          if (ph.visc_law == 1) mu = powf(T, (float)ph.visc_exp);
          const float div = du[0][0] + du[1][1] + du[2][2];
          const float vel[3] = {u, v, w};
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            if (kind == 1 && a != 0) continue;
            if (kind == 2 && a != 1) continue;
            const float ua = vel[a], mflux = rho * ua;
            float tau[3];
#pragma unroll
            for (int i2 = 0; i2 < 3; ++i2) tau[i2] = mu * (du[a][i2] + du[i2][a]);
            tau[a] -= (2.f / 3.f) * mu * div;
            const float qa = u * tau[0] + v * tau[1] + w * tau[2] + kap * mu * dT[a];
            float f[5];
            f[0] = -mflux;
            f[1] = -(mflux * u + (a == 0 ? p : 0.f)) + ire * tau[0];
            f[2] = -(mflux * v + (a == 1 ? p : 0.f)) + ire * tau[1];
            f[3] = -(mflux * w + (a == 2 ? p : 0.f)) + ire * tau[2];
            f[4] = -(et * ua + Href * ua) + ire * qa;
            if (a == 0) {
#pragma unroll
              for (int c = 0; c < 5; ++c) sFx[(c * FY + (bj - HB)) * (FX + 4) + (bi - HB + 2)] = f[c];
            } else if (a == 1) {
#pragma unroll
              for (int c = 0; c < 5; ++c) sFy[(c * (FY + 4) + (bj - HB + 2)) * FX + (bi - HB)] = f[c];
            } else {
#pragma unroll
              for (int c = 0; c < 5; ++c) fz[c] = f[c];
            }
          }
        };
        point(HB + tx, HB + ty, 0);
        // strip points: 4 columns x FY rows (x strips) and 4 rows x FX columns (y strips), spread
        // over all threads of the CTA
        for (int e = tid; strips && e < 4 * (FX + FY); e += NT) {
          if (e < 4 * FY) {
            const int col = e % 4, row = e / 4;
            point(col < 2 ? (HB - 2 + col) : (HB + FX + col - 2), HB + row, 1);
          } else {
            const int e2 = e - 4 * FY, col = e2 % FX, r4 = e2 / FX;
            point(HB + col, r4 < 2 ? (HB - 2 + r4) : (HB + FY + r4 - 2), 2);
          }
        }
        __syncthreads();
        // queues: Phi_z of planes G-4..G, dt (Dx Phi_x + Dy Phi_y) of planes G-2..G
#pragma unroll
        for (int c = 0; c < 5; ++c) {
#pragma unroll
          for (int a = 0; a < 4; ++a) phiz[a][c] = phiz[a + 1][c];
          phiz[4][c] = fz[c];
          rxy[0][c] = rxy[1][c];
          rxy[1][c] = rxy[2][c];
          float r = 0.f;
          if (strips) {
            const float* Fx = sFx + (c * FY + ty) * (FX + 4) + tx + 2;
            const float* Fy = sFy + (c * (FY + 4) + ty + 2) * FX + tx;
            r = k1x * (Fx[1] - Fx[-1]) + k2x * (Fx[2] - Fx[-2]);
            r = fmaf(k1y, Fy[FX] - Fy[-FX], r);
            r = fmaf(k2y, Fy[2 * FX] - Fy[-2 * FX], r);
          }
          rxy[2][c] = r;
        }
        // output plane z = G - 2
        const int z = G - 2;
        const int lx = tx0 + tx, ly = ty0 + ty;
        if (z >= z0 && z < z1 && lx < d.sx && ly < d.sy) {
          const long long gi = d.bbase + (long long)(d.ox + lx) + (long long)d.bnx * ((long long)(d.oy + ly) + (long long)d.bny * (d.oz + z));
#pragma unroll
          for (int c = 0; c < 5; ++c) {
            float r = rxy[0][c];
            r = fmaf(k1z, phiz[3][c] - phiz[1][c], r);
            r = fmaf(k2z, phiz[4][c] - phiz[0][c], r);
            const double dtR = (double)r;
            const double qn = first ? dtR : fma(A, Q[c * d.bN + gi], dtR);
            if (!last) Q[c * d.bN + gi] = qn;
            Uout[c * d.bN + gi] = fma(B, qn, Uin[c * d.bN + gi]);
          }
        }
      }
      __syncthreads();
    }
  }
}

// ------------------------------------------------------------------------------- launchers

int fused_smem_bytes(int fy) {
  if (fy == 4) return (int)FusedSmem<32, 4>::bytes;
  if (fy == 16) return (int)FusedSmem<32, 16>::bytes;
  return (int)FusedSmem<32, 8>::bytes;
}

int launch_halo_prims(const Geometry& g, const Physics& ph, const StepSched& sc, const double* ring, const SubDev* subs,
                      const int* halo, long long nhalo, float* Wh, int s, void* stream, long long* launches,
                      const Timer* tm) {
  cudaStream_t st = (cudaStream_t)stream;
  if (nhalo <= 0) return 0;
  if (tm) tm->rec(tm->self, 0, 1);
  k_halo_prims<<<(unsigned)((nhalo + 255) / 256), 256, 0, st>>>(g, ph, sc, ring, subs, (const int2*)halo, nhalo, Wh, s);
  if (tm) tm->rec(tm->self, 0, 0);
  if (launches) *launches += 1;
  return (int)cudaGetLastError();
}

template <int FX, int FY>
static int fused_impl(const Geometry& g, const Physics& ph, const StepSched& sc, const FusedLaunch& a, cudaStream_t st) {
  const size_t sm = FusedSmem<FX, FY>::bytes;
  static bool attr_set = false;  // per process: the attribute is a property of the kernel
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_stage_fused<FX, FY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return (int)e;
    attr_set = true;
  }
  k_stage_fused<FX, FY><<<a.grid, FX * FY, sm, st>>>(g, ph, sc, a.Uin, a.Uout, a.ring, a.in_ring, a.out_ring, a.Q,
                                                    a.subs, a.work, a.nwork, a.Wh, a.stage, a.A, a.B, a.dt, a.first,
                                                    a.last);
  return (int)cudaGetLastError();
}

int launch_stage_fused(const Geometry& g, const Physics& ph, const StepSched& sc, const FusedLaunch& a, void* stream,
                       long long* launches, const Timer* tm) {
  cudaStream_t st = (cudaStream_t)stream;
  if (tm) tm->rec(tm->self, 2, 1);
  int rc;
  if (a.fy == 4) rc = fused_impl<32, 4>(g, ph, sc, a, st);
  else if (a.fy == 16) rc = fused_impl<32, 16>(g, ph, sc, a, st);
  else rc = fused_impl<32, 8>(g, ph, sc, a, st);
  if (tm) tm->rec(tm->self, 2, 0);
  if (launches) *launches += 1;
  return rc;
}

}  // namespace cfs
