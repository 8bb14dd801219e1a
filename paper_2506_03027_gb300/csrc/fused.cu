// fused.cu -- fused LSERK stage for the FP32-intermediate form (3-D Navier-Stokes, CD4/AT4).
//
// One launch per RK stage (Eq. 3) does what k_view + k_flux + k_rk do in three: each CTA owns an
// FX x FY column tile of one sub-domain and marches through its z-planes.  Per plane L:
//   stage  L + 1         asynchronous copies (cp.async) of the raw stage input of the next plane
//                        -- FP64 conserved values of own points and synchronous halos, FP32
//                        primitives of AT/AS halo points from the per-step halo store
//                        (k_halo_prims) -- into a staging buffer, overlapping the work below;
//   convert L            staging -> FP32 primitives: u, v, w, T into a five-plane ring (the CD4
//                        gradient stencil in z), rho, p', et' into a three-plane ring over the
//                        tile and its 2-wide strips (values at flux points only);
//   plane G = L - 2      CD4 gradients, viscous stresses and heat flux (Eq. A3-A4), combined
//                        fluxes Phi_a = -F_a + Fv_a / Re (Eq. A2); Phi_x, Phi_y of the tile and
//                        its x / y strips to shared memory, Phi_z of the tile in registers;
//   accumulate           dt R of the tile column is gathered in a queue of four planes: Phi_z of
//                        plane G contributes to planes G-2..G+2 (CD4 in z), dt (D_x Phi_x +
//                        D_y Phi_y) to plane G;
//   plane z = G - 2      complete: FP64 low-storage update Q = A Q + dt R, U^(m) = U^(m-1) + B Q.
// Conversions between FP64 and FP32 use the integer-pipe routines of device_common.cuh.
// k_halo_prims runs once per asynchronous step: for every halo point a sub-domain reads from a
// neighbour it applies the AT weights of all s stages to the C delayed levels in FP64 (Eq. 14-15
// and the buffer updates of Eq. 8 / Table 5) and stores the FP32 primitives per stage.
#include <cuda_runtime.h>

#include "cfs_internal.h"
#include "device_common.cuh"

namespace cfs {

namespace {

constexpr int HB = 4;  // halo of the box: 2r for the viscous CD4 operator

// FP32 copies of the physical constants, converted once per thread.
struct Phys32 {
  float gm1, gM2, ire, kap, Href, Eh, El, vexp;
  int law;
};

__device__ __forceinline__ Phys32 phys32(const Physics& ph) {
  Phys32 q;
  q.gm1 = (float)ph.gm1;
  q.gM2 = (float)ph.gM2;
  q.ire = (float)ph.ire;
  q.kap = (float)ph.kappa;
  q.Href = (float)ph.H_ref;
  q.Eh = (float)ph.E_ref;
  q.El = (float)(ph.E_ref - (double)q.Eh);
  q.vexp = (float)ph.visc_exp;
  q.law = ph.visc_law;
  return q;
}

// FP32 primitives (rho, u, v, w, p - p_ref, T, rho E + p - H_ref) from an FP64 conserved state
// (App. A; p and rho E carried as deviations from the reference state p_ref = 1/(gamma M^2),
// E_ref = p_ref/(gamma-1), so that FP32 rounding acts on O(1) deviations).
__device__ __forceinline__ void prims32(const double* u, const Phys32& k, float* w) {
  const float rho = d2f_fast(u[0]);
  const float ir = __fdividef(1.0f, rho);
  const float mx = d2f_fast(u[1]), my = d2f_fast(u[2]), mz = d2f_fast(u[3]);
  const float uu = mx * ir, vv = my * ir, ww = mz * ir;
  const float ke = 0.5f * (mx * uu + my * vv + mz * ww);
  const float rE = dev_fast(u[4], k.Eh, k.El);
  const float p = k.gm1 * (rE - ke);
  w[0] = rho;
  w[1] = uu;
  w[2] = vv;
  w[3] = ww;
  w[4] = p;
  w[5] = (k.gM2 * p + 1.0f) * ir;  // T
  w[6] = rE + p;                   // rho E + p - H_ref
}

}  // namespace

// ------------------------------------------------------------------------------- k_halo_prims

template <int S>
__global__ void __launch_bounds__(256) k_halo_prims(Geometry g, Physics ph, StepSched sc, const double* __restrict__ ring,
                                                    const SubDev* __restrict__ subs, const int2* __restrict__ halo,
                                                    long long nhalo, float* __restrict__ Wh) {
  sc = resolve(sc);
  if (sc.mode == 0) return;  // synchronous step: no halo store is read
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nhalo) return;
  const Phys32 k32 = phys32(ph);
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
#pragma unroll
    for (int v = 0; v < 5; ++v) u[v] = src[v * d.bN + gi];
    float w[7];
    prims32(u, k32, w);
#pragma unroll
    for (int c = 0; c < 7; ++c) Wh[(long long)c * P + o] = w[c];
    return;
  }
  // AT: U_buf^(m) = sum_l W^(m)_l(k) U^{n-k-l} for every stage m, accumulated in FP64; with the
  // learned halo, face points start from the network's stage-0 value and add (W^(m) - W^(0)) R
  const bool learned = sc.LH && ((int)(ci < 0 || ci >= d.sx) + (int)(cj < 0 || cj >= d.sy) + (int)(ck < 0 || ck >= d.sz) == 1);
  double acc[S][5];
#pragma unroll
  for (int m = 0; m < S; ++m)
#pragma unroll
    for (int v = 0; v < 5; ++v) acc[m][v] = learned ? sc.LH[(long long)v * g.Ptot + d.pbase + t] : 0.0;
  for (int l = 0; l < sc.C; ++l) {
    const double* src = ring + (long long)((sc.n - kd - l) % sc.R) * lvN;
    double r[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) r[v] = src[v * d.bN + gi];
    const double w0 = learned ? __ldg(sc.W + (kd * S) * sc.C + l) : 0.0;
#pragma unroll
    for (int m = 0; m < S; ++m) {
      if (learned && m == 0) continue;
      const double wl = __ldg(sc.W + (kd * S + m) * sc.C + l) - w0;
#pragma unroll
      for (int v = 0; v < 5; ++v) acc[m][v] = fma(wl, r[v], acc[m][v]);
    }
  }
#pragma unroll
  for (int m = 0; m < S; ++m) {
    float w[7];
    prims32(acc[m], k32, w);
#pragma unroll
    for (int c = 0; c < 7; ++c) Wh[(long long)(m * 7 + c) * P + o] = w[c];
  }
}

// ------------------------------------------------------------------------------- k_stage_fused

template <int FX, int FY>
struct FusedSmem {
  static constexpr int BX = FX + 2 * HB, BY = FY + 2 * HB, NB = BX * BY;  // box: tile + halo of 4
  static constexpr int WX = FX + 4, WY = FY + 4, NW = WX * WY;            // window: tile + strips of 2
  static constexpr int STG = 2 * 5 * NB;                                  // staging, 5 x 8 bytes per box point
  static constexpr int R4 = 5 * 4 * NB;   // u, v, w, T of planes G-2..G+2
  static constexpr int R3 = 3 * 3 * NW;   // rho, p', et' of planes G..G+2 on the window
  static constexpr int FXS = 5 * FY * (FX + 4);  // Phi_x of tile + x strips
  static constexpr int FYS = 5 * (FY + 4) * FX;  // Phi_y of tile + y strips
  static constexpr size_t bytes = sizeof(float) * (STG + R4 + R3 + FXS + FYS);
};

// Where the stage input of a box point comes from: the FP64 state (own points, synchronous halos,
// and box points no output depends on) or the per-step halo store.  dx, dy, dz: distance outside
// the sub-domain along each axis.  The sub-domain's view holds faces up to depth HB and edges up
// to r x r; a narrow ragged tile's box reaches further, and those points feed no output.
__device__ __forceinline__ bool from_store(int mode, int r, int dx, int dy, int dz) {
  const int nout = (dx > 0) + (dy > 0) + (dz > 0);
  const bool inview = (nout == 1 && dx <= HB && dy <= HB && dz <= HB) || (nout == 2 && dx <= r && dy <= r && dz <= r);
  return mode != 0 && nout > 0 && inview;
}

// Per-thread description of the box columns (i, j) it loads on every plane of a work item.
template <int KB>
struct BoxCols {
  int xy[KB];   // gx + bnx gy of the wrapped in-block position
  int pxy[KB];  // (lx + G) + ex (ly + G) in the padded box
  int dxy[KB];  // dx | dy << 8 (distance outside the sub-domain), -1 for no column
};

template <int FX, int FY>
__global__ void __launch_bounds__(FX* FY, (FX * FY >= 512) ? 1 : 2) k_stage_fused(Geometry g, Physics ph, StepSched sc,
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
  constexpr int BX = S::BX, NB = S::NB, WX = S::WX, NW = S::NW, NT = FX * FY;
  extern __shared__ __align__(16) float smem[];
  double* sStg = reinterpret_cast<double*>(smem);  // [5][NB] FP64, or FP32 pairs for halo points
  float* sStgF = smem;
  float* sR4 = smem + S::STG;
  float* sR3 = sR4 + S::R4;
  float* sFx = sR3 + S::R3;
  float* sFy = sFx + S::FXS;
  const int tid = threadIdx.x, tx = tid % FX, ty = tid / FX;
  constexpr int KB = (NB + NT - 1) / NT;
  // constants converted from FP64 once per CTA (physics) and once per work item (dt x CD
  // coefficients) by one thread; the work-item set is double-buffered by parity so that thread
  // can run ahead of the others by one item
  __shared__ Phys32 sPh;
  __shared__ float sK[2][12];
  if (tid == 0) sPh = phys32(ph);
  __syncthreads();
  const Phys32 k32 = sPh;
  const long long P = g.Ptot;
  const float* __restrict__ WhS = Wh + (long long)((sc.mode == 2) ? 0 : stage) * 7 * P;

  for (int wi = blockIdx.x, par = 0; wi < nwork; wi += gridDim.x, par ^= 1) {
    const int* wk = work + 4 * wi;  // (sub-domain, x0, y0, z0 | z1 << 16)
    const SubDev d = subs[wk[0]];
    const int tx0 = wk[1], ty0 = wk[2];
    const int z0 = wk[3] & 0xffff, z1 = wk[3] >> 16;  // output planes [z0, z1) of the sub-domain
    if (tid == 0) {
      for (int a = 0; a < 3; ++a) {
        sK[par][a] = (float)d.c1[a];
        sK[par][3 + a] = (float)d.c2[a];
        sK[par][6 + a] = (float)(dt * d.c1[a]);
        sK[par][9 + a] = (float)(dt * d.c2[a]);
      }
    }
    BoxCols<KB> bc;
#pragma unroll
    for (int k = 0; k < KB; ++k) {
      const int p = tid + k * NT;
      bc.dxy[k] = -1;
      if (p < NB) {
        const int lx = tx0 - HB + p % BX, ly = ty0 - HB + p / BX;
        const int dx = lx < 0 ? -lx : (lx >= d.sx ? lx - d.sx + 1 : 0);
        const int dy = ly < 0 ? -ly : (ly >= d.sy ? ly - d.sy + 1 : 0);
        bc.xy[k] = wrapc(d.ox + lx, d.bnx) + d.bnx * wrapc(d.oy + ly, d.bny);
        bc.pxy[k] = (lx + g.G) + d.ex * (ly + g.G);
        bc.dxy[k] = dx | (dy << 8);
      }
    }
    // dt R of the tile column for planes G-2..G+1 (before the contributions of flux plane G)
    float acc[4][5];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 5; ++c) acc[a][c] = 0.f;

    // plane-dependent parts of the source offsets
    auto plane_src = [&](int L, long long& zoff, long long& pz, int& dz) {
      dz = L < 0 ? -L : (L >= d.sz ? L - d.sz + 1 : 0);
      zoff = d.bbase + (long long)d.bnx * d.bny * wrapc(d.oz + L, d.bnz);
      pz = d.pbase + (long long)d.ex * d.ey * (L + g.Gz);
    };
    auto issue = [&](int L) {
      long long zoff, pz;
      int dz;
      plane_src(L, zoff, pz, dz);
#pragma unroll
      for (int k = 0; k < KB; ++k) {
        const int p = tid + k * NT;
        if (bc.dxy[k] < 0) continue;
        if (!from_store(sc.mode, g.r, bc.dxy[k] & 255, bc.dxy[k] >> 8, dz)) {
          const double* src = Uin + zoff + bc.xy[k];
#pragma unroll
          for (int v = 0; v < 5; ++v) cp_async8(sStg + v * NB + p, src + v * d.bN);
        } else {
          const float* src = WhS + pz + bc.pxy[k];
#pragma unroll
          for (int c = 0; c < 7; ++c) cp_async4(sStgF + 2 * ((c >> 1) * NB + p) + (c & 1), src + (long long)c * P);
        }
      }
      cp_async_commit();
    };

    issue(z0 - HB);
    for (int L = z0 - HB; L < z1 + HB; ++L) {
      // ---- staged plane L -> primitives in the rings
      cp_async_wait_all();
      __syncthreads();
      {
        float* r4 = sR4 + ((L + 15) % 5) * 4 * NB;
        float* r3 = sR3 + ((L + 15) % 3) * 3 * NW;
        const int dz = L < 0 ? -L : (L >= d.sz ? L - d.sz + 1 : 0);
#pragma unroll
        for (int k = 0; k < KB; ++k) {
          const int p = tid + k * NT;
          if (bc.dxy[k] < 0) continue;
          float w[7];
          if (!from_store(sc.mode, g.r, bc.dxy[k] & 255, bc.dxy[k] >> 8, dz)) {
            double u[5];
#pragma unroll
            for (int v = 0; v < 5; ++v) u[v] = sStg[v * NB + p];
            prims32(u, k32, w);
          } else {
#pragma unroll
            for (int c = 0; c < 7; ++c) w[c] = sStgF[2 * ((c >> 1) * NB + p) + (c & 1)];
          }
          r4[p] = w[1];
          r4[NB + p] = w[2];
          r4[2 * NB + p] = w[3];
          r4[3 * NB + p] = w[5];
          const int wi2 = p % BX - (HB - 2), wj2 = p / BX - (HB - 2);
          if (wi2 >= 0 && wi2 < WX && wj2 >= 0 && wj2 < S::WY) {
            const int qw = wj2 * WX + wi2;
            r3[qw] = w[0];
            r3[NW + qw] = w[4];
            r3[2 * NW + qw] = w[6];
          }
        }
      }
      __syncthreads();
      if (L + 1 < z1 + HB) issue(L + 1);

      const int G = L - 2;
      if (G < z0 - 2 || G > z1 + 1) continue;
      const float c1x = sK[par][0], c1y = sK[par][1], c1z = sK[par][2];
      const float c2x = sK[par][3], c2y = sK[par][4], c2z = sK[par][5];
      const float k1x = sK[par][6], k1y = sK[par][7], k1z = sK[par][8];
      const float k2x = sK[par][9], k2y = sK[par][10], k2z = sK[par][11];
      // ---- stage input and Q of the output plane z = G - 2 (in flight during the flux work)
      const int z = G - 2;
      const int lx = tx0 + tx, ly = ty0 + ty;
      const bool outp = z >= z0 && z < z1 && lx < d.sx && ly < d.sy;
      long long go = 0;
      double uin[5], qin[5];
      if (outp) {
        go = d.bbase + (long long)(d.ox + lx) + (long long)d.bnx * ((long long)(d.oy + ly) + (long long)d.bny * (d.oz + z));
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          uin[c] = Uin[c * d.bN + go];
          qin[c] = first ? 0.0 : Q[c * d.bN + go];
        }
      }
      // ---- fluxes of plane G
      const float* pl[5];
#pragma unroll
      for (int o = 0; o < 5; ++o) pl[o] = sR4 + ((G - 2 + o + 15) % 5) * 4 * NB;  // planes G-2..G+2
      const float* r3c = sR3 + ((G + 15) % 3) * 3 * NW;
      const bool strips = (G >= z0 && G < z1);
      float fz[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
      // one gradient/flux evaluation at box point (bi, bj) of plane G: kind 0 tile point (Phi_x,
      // Phi_y to shared memory, Phi_z to registers), 1 x-strip (Phi_x), 2 y-strip (Phi_y)
      auto point = [&](int bi, int bj, int kind) {
        const float* P0 = pl[2];
        const int q = bj * BX + bi;
        const int qw = (bj - (HB - 2)) * WX + (bi - (HB - 2));
        float du[3][3], dT[3];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const float* f = P0 + v * NB;
          const float gx_ = c1x * (f[q + 1] - f[q - 1]) + c2x * (f[q + 2] - f[q - 2]);
          const float gy_ = c1y * (f[q + BX] - f[q - BX]) + c2y * (f[q + 2 * BX] - f[q - 2 * BX]);
          const float gz_ = c1z * (pl[3][v * NB + q] - pl[1][v * NB + q]) + c2z * (pl[4][v * NB + q] - pl[0][v * NB + q]);
          if (v < 3) { du[v][0] = gx_; du[v][1] = gy_; du[v][2] = gz_; }
          else { dT[0] = gx_; dT[1] = gy_; dT[2] = gz_; }
        }
        const float u = P0[q], v = P0[NB + q], w = P0[2 * NB + q], T = P0[3 * NB + q];
        const float rho = r3c[qw], p = r3c[NW + qw], et = r3c[2 * NW + qw];
        float mu = 1.f;
        if (k32.law == 1) mu = powf(T, k32.vexp);
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
          const float qa = u * tau[0] + v * tau[1] + w * tau[2] + k32.kap * mu * dT[a];
          float f[5];
          f[0] = -mflux;
          f[1] = -(mflux * u + (a == 0 ? p : 0.f)) + k32.ire * tau[0];
          f[2] = -(mflux * v + (a == 1 ? p : 0.f)) + k32.ire * tau[1];
          f[3] = -(mflux * w + (a == 2 ? p : 0.f)) + k32.ire * tau[2];
          f[4] = -(et * ua + k32.Href * ua) + k32.ire * qa;
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
      // ---- dt R queue: Phi_z(G) enters planes G-2..G+2 with the CD4 weights, the in-plane
      // divergence enters plane G; plane G-2 is then complete
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        float r = 0.f;
        if (strips) {
          const float* Fx = sFx + (c * FY + ty) * (FX + 4) + tx + 2;
          const float* Fy = sFy + (c * (FY + 4) + ty + 2) * FX + tx;
          r = k1x * (Fx[1] - Fx[-1]) + k2x * (Fx[2] - Fx[-2]);
          r = fmaf(k1y, Fy[FX] - Fy[-FX], r);
          r = fmaf(k2y, Fy[2 * FX] - Fy[-2 * FX], r);
        }
        const float out = fmaf(k2z, fz[c], acc[0][c]);
        acc[0][c] = fmaf(k1z, fz[c], acc[1][c]);
        acc[1][c] = acc[2][c] + r;
        acc[2][c] = fmaf(-k1z, fz[c], acc[3][c]);
        acc[3][c] = -k2z * fz[c];
        if (outp) {
          const double dtR = f2d_fast(out);
          const double qn = first ? dtR : fma(A, qin[c], dtR);
          if (!last) Q[c * d.bN + go] = qn;
          Uout[c * d.bN + go] = fma(B, qn, uin[c]);
        }
      }
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
  const unsigned nb = (unsigned)((nhalo + 255) / 256);
  if (tm) tm->rec(tm->self, 0, 1);
  if (s == 2) k_halo_prims<2><<<nb, 256, 0, st>>>(g, ph, sc, ring, subs, (const int2*)halo, nhalo, Wh);
  else k_halo_prims<5><<<nb, 256, 0, st>>>(g, ph, sc, ring, subs, (const int2*)halo, nhalo, Wh);
  if (tm) tm->rec(tm->self, 0, 0);
  if (launches) *launches += 1;
  return (int)cudaGetLastError();
}

template <int FX, int FY>
static int fused_prepare(int* blocks_per_sm) {
  const size_t sm = FusedSmem<FX, FY>::bytes;
  static bool attr_set = false;  // per process: the attribute is a property of the kernel
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_stage_fused<FX, FY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return (int)e;
    attr_set = true;
  }
  if (blocks_per_sm) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_stage_fused<FX, FY>, FX * FY, sm);
    if (e != cudaSuccess) return (int)e;
  }
  return 0;
}

int fused_blocks_per_sm(int fy, int* blocks) {
  if (fy == 4) return fused_prepare<32, 4>(blocks);
  if (fy == 16) return fused_prepare<32, 16>(blocks);
  return fused_prepare<32, 8>(blocks);
}

template <int FX, int FY>
static int fused_impl(const Geometry& g, const Physics& ph, const StepSched& sc, const FusedLaunch& a, cudaStream_t st) {
  const int rc = fused_prepare<FX, FY>(nullptr);
  if (rc) return rc;
  k_stage_fused<FX, FY><<<a.grid, FX * FY, FusedSmem<FX, FY>::bytes, st>>>(
      g, ph, sc, a.Uin, a.Uout, a.ring, a.in_ring, a.out_ring, a.Q, a.subs, a.work, a.nwork, a.Wh, a.stage, a.A, a.B,
      a.dt, a.first, a.last);
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
