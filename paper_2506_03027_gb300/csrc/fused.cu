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
// neighbour it applies the AT weights of all s stages to the C delayed levels (Eq. 14-15 and the
// buffer updates of Eq. 8 / Table 5) -- FP32 sums over the levels' differences from the newest
// level, in FP64 for the gather entries of connected grids -- and stores the FP32 primitives per
// stage.
#include <cuda_runtime.h>

#include <mutex>

#include "cfs_internal.h"
#include "device_common.cuh"

namespace cfs {

namespace {

constexpr int HB = 4;  // halo of the box: 2r for the viscous CD4 operator
constexpr unsigned STG_WAIT_LIMIT = 1u << 20;  // polls of the staging mbarrier before giving up

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// Every thread of the CTA arrives on the staging barrier once per plane, announcing the bytes of
// the bulk copy it is about to issue (0: none).
__device__ __forceinline__ void stg_arrive(unsigned long long* bar, unsigned tx) {
  if (tx) asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(tx) : "memory");
  else asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_addr(bar)) : "memory");
}

// One row of FP64 values global -> shared by the bulk-copy engine, completing on the barrier
// (both addresses 16-byte aligned, bytes a multiple of 16).
__device__ __forceinline__ void stg_bulk(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

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

// FP32 primitives (rho, u, v, w, p - p_ref, T, rho E + p - H_ref) from the FP32 conserved values
// rho, rho u, rho v, rho w and the deviation rho E - E_ref (App. A; p and rho E carried as
// deviations from the reference state p_ref = 1/(gamma M^2), E_ref = p_ref/(gamma-1), so that FP32
// rounding acts on O(1) deviations).
__device__ __forceinline__ void prims32f(float rho, float mx, float my, float mz, float rE, const Phys32& k, float* w) {
  const float ir = __fdividef(1.0f, rho);
  const float uu = mx * ir, vv = my * ir, ww = mz * ir;
  const float ke = 0.5f * (mx * uu + my * vv + mz * ww);
  const float p = k.gm1 * (rE - ke);
  w[0] = rho;
  w[1] = uu;
  w[2] = vv;
  w[3] = ww;
  w[4] = p;
  w[5] = (k.gM2 * p + 1.0f) * ir;  // T
  w[6] = rE + p;                   // rho E + p - H_ref
}

// The same from an FP64 conserved state.
__device__ __forceinline__ void prims32(const double* u, const Phys32& k, float* w) {
  prims32f(d2f_fast(u[0]), d2f_fast(u[1]), d2f_fast(u[2]), d2f_fast(u[3]), dev_fast(u[4], k.Eh, k.El), k, w);
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
  const int t = hv.y;  // index in the sub-domain's padded box (32-bit)
  const SubDev d = subs[sid];
  const int exy = d.ex * d.ey;
  const int k = t / exy, r2 = t - k * exy, j = r2 / d.ex, i = r2 - j * d.ex;
  const int ci = i - g.G, cj = j - g.G, ck = k - g.Gz;
  // halo points lie within G of the sub-domain: one conditional wrap per axis
  auto wrap1 = [](int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); };
  const int gx = wrap1(d.ox + ci, d.bnx), gy = wrap1(d.oy + cj, d.bny), gz = wrap1(d.oz + ck, d.bnz);
  const long long gi = d.bbase + (long long)gx + (long long)d.bnx * ((long long)gy + (long long)d.bny * gz);
  const long long lvN = 5 * g.N, P = g.Ptot, o = d.pbase + t;
  const int ux = d.ox + ci, uy = d.oy + cj;
  const bool gather = d.ebase >= 0 && (ux < 0 || ux >= d.bnx || uy < 0 || uy >= d.bny);
  // delay of the faces the point lies beyond (faces on a physical boundary of the block: none)
  int kd = 0;
  if ((ci < 0 || ci >= d.sx) && !(gather && ((d.phys >> (ci < 0 ? 0 : 1)) & 1))) kd = max(kd, face_delay(sc, sid, ci < 0 ? 0 : 1));
  if ((cj < 0 || cj >= d.sy) && !(gather && ((d.phys >> (cj < 0 ? 2 : 3)) & 1))) kd = max(kd, face_delay(sc, sid, cj < 0 ? 2 : 3));
  if (ck < 0 || ck >= d.sz) kd = max(kd, face_delay(sc, sid, ck < 0 ? 4 : 5));
  // ring slot of level n - kd - l: (n mod R) - kd - l, wrapped once (kd + l < R)
  const int nR = (int)(sc.n % sc.R);
  auto slot = [&](int l) { const int q = nR - kd - l; return q < 0 ? q + sc.R : q; };
  if (gather) {
    // beyond a non-periodic block face (a connected grid): the gather entry's sources.  Entries
    // whose sources are the sub-domain's own points (wall mirrors, outflow copies) take the
    // current stage values inside the fused stage; the others -- neighbouring PEs' values seen
    // with the delay of the faces crossed, and far-field constants -- are prepared here per stage
    // as for any other halo point.
    const GatherEntry& E = g.gent[g.emap[d.ebase + (ux + g.GE) + (long long)d.gmx * ((uy + g.GE) + (long long)d.gmy * gz)]];
    // (own sources beyond the sub-domain in z are reached across the periodic wrap: foreign,
    // prepared here like any other; the fused stage reads them from this store)
    if (E.nt == 1 && !(E.flags[0] & 2) && E.sid[0] == sid && ck >= 0 && ck < d.sz) return;
    double acc[S][5];
#pragma unroll
    for (int m = 0; m < S; ++m)
#pragma unroll
      for (int v = 0; v < 5; ++v) acc[m][v] = E.cst[v];
    for (int q = 0; q < E.nt; ++q) {
      const double wt = E.w[q], wf = (E.flags[q] & 1) ? -wt : wt;
      const long long so = E.off[q], sbN = E.bN[q];
      for (int l = 0; l < (sc.mode == 2 ? 1 : sc.C); ++l) {
        const double* src = ring + (long long)slot(l) * lvN;
        double r[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) r[v] = src[so + v * sbN];
#pragma unroll
        for (int m = 0; m < S; ++m) {
          const double wl = sc.mode == 2 ? 1.0 : __ldg(sc.W + (kd * S + m) * sc.C + l);
#pragma unroll
          for (int v = 0; v < 5; ++v) acc[m][v] = fma(((v >= 1 && v <= 3) ? wf : wt) * wl, r[v], acc[m][v]);
        }
      }
    }
#pragma unroll
    for (int m = 0; m < (sc.mode == 2 ? 1 : S); ++m) {
      float w[7];
      prims32(acc[m], k32, w);
#pragma unroll
      for (int c = 0; c < 7; ++c) Wh[(long long)(m * 7 + c) * P + o] = w[c];
    }
    return;
  }
  if (sc.mode == 2) {  // AS: the latest visible level, the same for every stage
    const double* src = ring + (long long)slot(0) * lvN;
    double u[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) u[v] = src[v * d.bN + gi];
    float w[7];
    prims32(u, k32, w);
#pragma unroll
    for (int c = 0; c < 7; ++c) Wh[(long long)c * P + o] = w[c];
    return;
  }
  // AT: U_buf^(m) = sum_l W^(m)_l(k) U^{n-k-l} for every stage m, written as
  // S_m U_0 + sum_{l>=1} W^(m)_l (U_l - U_0) with U_l = U^{n-k-l} and S_m = sum_l W^(m)_l, which is 1
  // up to the rounding of the table (the stage-0 extrapolation weights reproduce constants, the
  // derivative weights the later stages add sum to zero), and evaluated without FP64 arithmetic:
  // - each difference U_l - U_0 as an exact pair of floats: U_l = h + r (split_fast: h its FP32
  //   truncation), U_0 = h0 + l0, (h - h0) exact when the levels are within a factor of two;
  // - the weights as pairs of floats (table W32: S_m - 1, then W^(m)_1 .. W^(m)_{C-1});
  // - products of the high parts split exactly with an FMA and summed with TwoSum: the weights
  //   of large delays alternate in sign (sum |W| about 1,400 at k = 4 against 1 for the result),
  //   so plain FP32 sums would lose that factor; compensated, the sum has the accuracy of the
  //   FP64 one before its final rounding to the FP32 primitives.
  // With the learned halo, face points start from the network's stage-0 value and add the same
  // sums with W^(m) - W^(0) (table W32d).
  const bool learned = sc.LH && ((int)(ci < 0 || ci >= d.sx) + (int)(cj < 0 || cj >= d.sy) + (int)(ck < 0 || ck >= d.sz) == 1);
  const int C = sc.C;
  double r[CFS_MAX_LEVELS][5];
#pragma unroll
  for (int l = 0; l < CFS_MAX_LEVELS; ++l)
    if (l < C) {
      const double* src = ring + (long long)slot(l) * lvN;
#pragma unroll
      for (int v = 0; v < 5; ++v) r[l][v] = src[v * d.bN + gi];
    }
  float h0[5], l0[5], ah[CFS_MAX_LEVELS][5], al[CFS_MAX_LEVELS][5];  // U_l - U_0 = ah[l] + al[l]
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    h0[v] = d2f_fast(r[0][v]);
    l0[v] = dev_fast(r[0][v], h0[v], 0.f);
  }
#pragma unroll
  for (int l = 1; l < CFS_MAX_LEVELS; ++l)
    if (l < C)
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        float h, q;
        split_fast(r[l][v], h, q);
        ah[l][v] = __fsub_rn(h, h0[v]);
        al[l][v] = __fsub_rn(q, l0[v]);
      }
  // the value the sums are added to: U_0, or the network's stage-0 value (rho, momenta as pairs
  // of floats, rho E as its deviation from E_ref)
  float bh[4], bl[4], be;
  if (learned) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const double x = sc.LH[(long long)v * g.Ptot + d.pbase + t];
      bh[v] = d2f_fast(x);
      bl[v] = dev_fast(x, bh[v], 0.f);
    }
    be = dev_fast(sc.LH[4LL * g.Ptot + d.pbase + t], k32.Eh, k32.El);
  } else {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      bh[v] = h0[v];
      bl[v] = l0[v];
    }
    be = dev_fast(r[0][4], k32.Eh, k32.El);
  }
  const float2* __restrict__ wt = (const float2*)(learned ? sc.W32d : sc.W32) + (long long)kd * S * C;
#pragma unroll
  for (int m = 0; m < S; ++m) {
    float2 c[CFS_MAX_LEVELS];
#pragma unroll
    for (int l = 0; l < CFS_MAX_LEVELS; ++l) c[l] = l < C ? __ldg(wt + m * C + l) : make_float2(0.f, 0.f);
    float dl[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      float sh = 0.f, st = __fmul_rn(c[0].x, h0[v]);  // running sum and its error terms
#pragma unroll
      for (int l = 1; l < CFS_MAX_LEVELS; ++l)
        if (l < C) {
          const float p = __fmul_rn(c[l].x, ah[l][v]);
          const float pe = __fmaf_rn(c[l].x, ah[l][v], -p);  // exact: p + pe = c.x * ah
          const float s2 = __fadd_rn(sh, p);                  // TwoSum(sh, p)
          const float bv = __fsub_rn(s2, sh);
          const float se = __fadd_rn(__fsub_rn(sh, __fsub_rn(s2, bv)), __fsub_rn(p, bv));
          sh = s2;
          st = __fadd_rn(st, __fadd_rn(se, pe));
          st = __fmaf_rn(c[l].x, al[l][v], st);
          st = __fmaf_rn(c[l].y, ah[l][v], st);
        }
      dl[v] = (learned && m == 0) ? 0.f : __fadd_rn(sh, st);
    }
    float w[7];
    prims32f(bh[0] + (bl[0] + dl[0]), bh[1] + (bl[1] + dl[1]), bh[2] + (bl[2] + dl[2]), bh[3] + (bl[3] + dl[3]),
             be + dl[4], k32, w);
#pragma unroll
    for (int c7 = 0; c7 < 7; ++c7) Wh[(long long)(m * 7 + c7) * P + o] = w[c7];
  }
}

// ------------------------------------------------------------------------------- k_stage_fused

template <int FX, int FY>
struct FusedSmem {
  static constexpr int NT = FX * FY;
  static constexpr int BX = FX + 2 * HB, BY = FY + 2 * HB, NB = BX * BY;  // box: tile + halo of 4
  static constexpr int WX = FX + 4, WY = FY + 4, NW = WX * WY;            // window: tile + strips of 2
  static constexpr int STG = 2 * 5 * NB;      // staging, 5 x 8 bytes per box point
  static constexpr int R4 = 4 * 5 * NB;       // float4 (u, v, w, T) of planes G-2..G+2 on the box
  static constexpr int R3 = 4 * 3 * NW;       // float4 (rho, p', et', -) of planes G..G+2 on the window
  static constexpr int FX4 = 4 * FY * (FX + 4), FX1 = FY * (FX + 4);  // Phi_x (components 0-3, 4)
  static constexpr int FY4 = 4 * (FY + 4) * FX, FY1 = (FY + 4) * FX;  // Phi_y
  static constexpr size_t bytes = sizeof(float) * (STG + R4 + R3 + FX4 + FX1 + FY4 + FY1);
  // curvilinear blocks (App. A): the window's metric terms xi^_x, xi^_y, eta^_x, eta^_y, zeta^_z
  // and J in FP32 (z-independent, loaded once per work item), after the arrays above
  static constexpr int MET = 6 * NW;
  static constexpr size_t bytes_curv = bytes + sizeof(float) * MET;
};

// The view of a sub-domain holds faces up to depth HB and edges up to r x r (corners unused).
__device__ __forceinline__ bool in_view(int r, int dx, int dy, int dz) {
  const int nout = (dx > 0) + (dy > 0) + (dz > 0);
  return (nout == 1 && dx <= HB && dy <= HB && dz <= HB) || (nout == 2 && dx <= r && dy <= r && dz <= r);
}

// Source of a box point on a plane: 0 skip (no output reads it), 1 the FP64 stage input (own
// points; every point in synchronous mode), 2 the per-step halo store.  dx, dy, dz: distance
// outside the sub-domain along each axis.
__device__ __forceinline__ int box_source(int mode, int r, int dx, int dy, int dz) {
  if (dx == 0 && dy == 0 && dz == 0) return 1;
  if (!in_view(r, dx, dy, dz)) return 0;
  return mode == 0 ? 1 : 2;
}

// Per-thread box columns (i, j) of a work item, loaded on every plane.
template <int KB>
struct BoxCols {
  int xy[KB];   // gx + bnx gy of the wrapped in-block position
  int pxy[KB];  // (lx + G) + ex (ly + G) in the padded box
  int dxy[KB];  // dx | dy << 8 (distance outside the sub-domain), -1 for no column
  int pq[KB];   // box index | window index << 16 (window index 0xffff: outside the window)
  // beyond a non-periodic block face (connected grids): 0 not such a column; 1 | src << 2 |
  // mirror << 18 a wall mirror / outflow copy of the sub-domain's own point at box index src on
  // the planes inside the sub-domain (current stage value, momentum negated when mirrored; on
  // planes beyond it in z the source is the z-neighbour's, as for 2); 2 a neighbouring PE's or
  // far-field value (the halo store on asynchronous steps, an inline gather on synchronous ones)
  int gm[KB];
};

__device__ __forceinline__ float2 lo2(const float4& a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ float2 hi2(const float4& a) { return make_float2(a.z, a.w); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }

// CD4 first derivative along one axis of (u, v) and (w, T) from the box values at offsets
// -2, -1, +1, +2: c1 (f+1 - f-1) + c2 (f+2 - f-2), packed FP32 pairs.
__device__ __forceinline__ void cd4_pair(const float4& m2, const float4& m1, const float4& p1, const float4& p2, float c1,
                                         float c2, float2& duv, float2& dwT) {
  duv = __ffma2_rn(bc2(c1), sub2(lo2(p1), lo2(m1)), __fmul2_rn(bc2(c2), sub2(lo2(p2), lo2(m2))));
  dwT = __ffma2_rn(bc2(c1), sub2(hi2(p1), hi2(m1)), __fmul2_rn(bc2(c2), sub2(hi2(p2), hi2(m2))));
}

// Fused stage.  Per CTA a tile of FX x FY columns of one sub-domain and a chunk of its z-planes;
// one thread per tile column.  Per plane L of the march: asynchronous copies of plane L + 1
// (FP64 state for own points, FP32 halo primitives from the store) run while plane L is
// converted into the rings and plane G = L - 2 is differentiated; the dt R queue of the column
// then completes plane G - 2, which takes its FP64 low-storage update.  Box columns are handed out
// in two lists (inside the sub-domain first, then halo columns) so that a warp takes one source;
// columns no output reads are not loaded.
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
  constexpr int FXW = FX + 4;
  extern __shared__ __align__(16) float smem[];
  double* sStg = reinterpret_cast<double*>(smem);  // [5][NB] FP64, or FP32 pairs for halo points
  float* sStgF = smem;
  float4* sR4 = reinterpret_cast<float4*>(smem + S::STG);   // [5][NB]
  float4* sR3 = reinterpret_cast<float4*>(smem + S::STG + S::R4);  // [3][NW]
  float4* sFx4 = reinterpret_cast<float4*>(smem + S::STG + S::R4 + S::R3);  // [FY][FX + 4]
  float* sFx1 = smem + S::STG + S::R4 + S::R3 + S::FX4;
  float4* sFy4 = reinterpret_cast<float4*>(sFx1 + S::FX1);  // [FY + 4][FX]
  float* sFy1 = sFx1 + S::FX1 + S::FY4;
  float* sMet = sFy1 + S::FY1;  // [6][NW], curvilinear blocks only
  __shared__ unsigned short sList[NB];  // box indices: columns inside the sub-domain, then halo columns
  __shared__ int sNlist;
  const int tid = threadIdx.x, tx = tid % FX, ty = tid / FX, lane = tid & 31;
  constexpr int KB = (NB + NT - 1) / NT;
  // constants converted from FP64 once per CTA (physics) and once per work item (dt x CD
  // coefficients) by one thread; the work-item set is double-buffered by parity so that thread
  // can run ahead of the others by one item
  __shared__ Phys32 sPh;
  __shared__ float sK[2][12];
  // staging barrier: NT arrivals per phase plus the bytes of the plane's bulk row copies
  __shared__ __align__(8) unsigned long long sBar;
  if (tid == 0) {
    sPh = phys32(ph);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(&sBar)), "r"(NT) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  unsigned stg_phase = 0;  // parity of the staging barrier's next phase
  const Phys32 k32 = sPh;
  const long long P = g.Ptot;
  const float* __restrict__ WhS = Wh + (long long)((sc.mode == 2) ? 0 : stage) * 7 * P;

  for (int wi = blockIdx.x, par = 0; wi < nwork; wi += gridDim.x, par ^= 1) {
    const int* wk = work + 4 * wi;  // (sub-domain, x0, y0, z0 | z1 << 16)
    const SubDev d = subs[wk[0]];
    const int tx0 = wk[1], ty0 = wk[2];
    const int z0 = wk[3] & 0xffff, z1 = wk[3] >> 16;  // output planes [z0, z1) of the sub-domain
    const int fxa = min(FX, d.sx - tx0), fya = min(FY, d.sy - ty0);  // the tile's own extent
    if (tid == 0) {
      for (int a = 0; a < 3; ++a) {
        sK[par][a] = (float)d.c1[a];
        sK[par][3 + a] = (float)d.c2[a];
        sK[par][6 + a] = (float)(dt * d.c1[a]);
        sK[par][9 + a] = (float)(dt * d.c2[a]);
      }
    }
    // ---- column lists (warp 0, ordered ballots): a box column is read by some output when it
    // lies in the tile +- 4 along one axis or in the tile +- 2 along both; outside the sub-domain
    // in x or y it must also be in the view (faces, r x r edges)
    __syncthreads();  // the previous item's lists (and metric window) are no longer read
    // curvilinear block: the metric terms of the window (tile + strips of 2), z-independent, and
    // J of this thread's own column in FP64 for the update
    const bool curv = d.mbase >= 0;
    double Jown = 1.0;
    if (curv) {
      for (int e = tid; e < NW; e += NT) {
        const int gxw = d.ox + tx0 - 2 + e % WX, gyw = d.oy + ty0 - 2 + e / WX;
        // window points of a partial tile can lie beyond the plane (extended by G): no output
        // reads their fluxes, give them zeros
        const bool in = gxw >= -g.G && gxw < d.bnx + g.G && gyw >= -g.G && gyw < d.bny + g.G;
        const double* M = g.metric + d.mbase + (long long)(gxw + g.G) + (long long)d.mx * (gyw + g.G);
#pragma unroll
        for (int k = 0; k < 5; ++k) sMet[k * NW + e] = in ? (float)M[(long long)k * d.mpl] : 0.f;
        sMet[5 * NW + e] = in ? (float)M[6 * d.mpl] : 0.f;
      }
      const int lxo = min(tx0 + tx, d.sx - 1), lyo = min(ty0 + ty, d.sy - 1);
      Jown = g.metric[d.mbase + 6 * d.mpl + (long long)(d.ox + lxo + g.G) + (long long)d.mx * (d.oy + lyo + g.G)];
    }
    if (tid < 32) {
      int n = 0;
      for (int pass = 0; pass < 2; ++pass) {
        for (int p0 = 0; p0 < NB; p0 += 32) {
          const int p = p0 + lane;
          bool take = false;
          if (p < NB) {
            const int ti = p % BX - HB, tj = p / BX - HB;
            const bool need = (tj >= 0 && tj < fya && ti >= -HB && ti < fxa + HB) ||
                              (ti >= 0 && ti < fxa && tj >= -HB && tj < fya + HB) ||
                              (ti >= -2 && ti < fxa + 2 && tj >= -2 && tj < fya + 2);
            const int lx = tx0 + ti, ly = ty0 + tj;
            const int dx = lx < 0 ? -lx : (lx >= d.sx ? lx - d.sx + 1 : 0);
            const int dy = ly < 0 ? -ly : (ly >= d.sy ? ly - d.sy + 1 : 0);
            const bool inner = dx == 0 && dy == 0;
            take = need && (pass == 0 ? inner : (!inner && in_view(g.r, dx, dy, 0)));
          }
          const unsigned m = __ballot_sync(0xffffffffu, take);
          if (take) sList[n + __popc(m & ((1u << lane) - 1u))] = (unsigned short)p;
          n += __popc(m);
        }
      }
      if (lane == 0) sNlist = n;
    }
    __syncthreads();
    const int nlist = sNlist;
    BoxCols<KB> bc;
#pragma unroll
    for (int k = 0; k < KB; ++k) {
      const int i = tid + k * NT;
      bc.dxy[k] = -1;
      if (i < nlist) {
        const int p = sList[i];
        const int lx = tx0 - HB + p % BX, ly = ty0 - HB + p / BX;
        const int dx = lx < 0 ? -lx : (lx >= d.sx ? lx - d.sx + 1 : 0);
        const int dy = ly < 0 ? -ly : (ly >= d.sy ? ly - d.sy + 1 : 0);
        bc.xy[k] = wrapc(d.ox + lx, d.bnx) + d.bnx * wrapc(d.oy + ly, d.bny);
        bc.pxy[k] = (lx + g.G) + d.ex * (ly + g.G);
        bc.dxy[k] = dx | (dy << 8);
        const int wi2 = p % BX - (HB - 2), wj2 = p / BX - (HB - 2);
        const int qw = (wi2 >= 0 && wi2 < WX && wj2 >= 0 && wj2 < S::WY) ? wj2 * WX + wi2 : 0xffff;
        bc.pq[k] = p | (qw << 16);
        bc.gm[k] = 0;
        const int ux = d.ox + lx, uy = d.oy + ly;
        if (d.ebase >= 0 && (ux < 0 || ux >= d.bnx || uy < 0 || uy >= d.bny)) {
          // the gather entry of this column (extruded blocks: its kind does not depend on z)
          const GatherEntry& E = g.gent[g.emap[d.ebase + (ux + g.GE) + (long long)d.gmx * ((uy + g.GE) + (long long)d.gmy * d.oz)]];
          bc.gm[k] = 2;
          if (E.nt == 1 && !(E.flags[0] & 2) && E.sid[0] == wk[0]) {
            const long long gi = E.off[0] - d.bbase;
            const int sxg = (int)(gi % d.bnx), syg = (int)((gi / d.bnx) % d.bny);
            const int bi = sxg - d.ox - (tx0 - HB), bj = syg - d.oy - (ty0 - HB);
            if (bi >= 0 && bi < BX && bj >= 0 && bj < S::BY) bc.gm[k] = 1 | ((bj * BX + bi) << 2) | ((E.flags[0] & 1) << 18);
          }
        }
      }
    }
    // dt R of the tile column for planes G-2..G+1 (before the contributions of flux plane G),
    // components (0, 1), (2, 3) as pairs and 4
    float2 aq[4][2];
    float aq4[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      aq[a][0] = make_float2(0.f, 0.f);
      aq[a][1] = make_float2(0.f, 0.f);
      aq4[a] = 0.f;
    }

    // plane-dependent parts of the source offsets
    auto plane_src = [&](int L, long long& zoff, long long& pz, int& dz) {
      dz = L < 0 ? -L : (L >= d.sz ? L - d.sz + 1 : 0);
      zoff = d.bbase + (long long)d.bnx * d.bny * wrapc(d.oz + L, d.bnz);
      pz = d.pbase + (long long)d.ex * d.ey * (L + g.Gz);
    };
    // On asynchronous steps the FP64 values come only from the sub-domain's own points: the rows
    // of the box inside the sub-domain, x in [lx0, lx1), y in [ly0, ly1), are contiguous in the
    // state and go as bulk row copies (when 16-byte aligned) instead of per-value copies.
    const int lx0 = max(tx0 - HB, 0), lx1 = min(tx0 + fxa + HB, d.sx);
    const int ly0 = max(ty0 - HB, 0), ly1 = min(ty0 + fya + HB, d.sy);
    const bool bulk = sc.mode != 0 && ((d.ox + lx0) & 1) == 0 && ((lx1 - lx0) & 1) == 0 && (d.bnx & 1) == 0 &&
                      (d.bbase & 1) == 0 && (d.bN & 1) == 0 && (g.N & 1) == 0;
    auto issue = [&](int L) {
      long long zoff, pz;
      int dz;
      plane_src(L, zoff, pz, dz);
      unsigned txb = 0;
      const double* bsrc = nullptr;
      double* bdst = nullptr;
      if (bulk && dz == 0 && tid < 5 * S::BY) {
        const int v = tid / S::BY, j = tid - v * S::BY, ly = ty0 - HB + j;
        if (ly >= ly0 && ly < ly1) {
          bsrc = Uin + zoff + (long long)v * d.bN + (long long)d.bnx * (d.oy + ly) + (d.ox + lx0);
          bdst = sStg + v * NB + j * BX + (lx0 - (tx0 - HB));
          txb = (unsigned)(lx1 - lx0) * 8u;
        }
      }
      if (txb) asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // after the generic reads of the buffer
      stg_arrive(&sBar, txb);
      if (txb) stg_bulk(bdst, bsrc, txb, &sBar);
#pragma unroll
      for (int k = 0; k < KB; ++k) {
        if (bc.dxy[k] < 0) continue;
        const int p = bc.pq[k] & 0xffff;
        const int src = box_source(sc.mode, g.r, bc.dxy[k] & 255, bc.dxy[k] >> 8, dz);
        if (src == 1 && bulk) continue;  // in a bulk row
        // a wall mirror's source is the own point of the same plane only inside the sub-domain in z;
        // beyond it in z the source belongs to the neighbouring PE in z (foreign)
        const int gmk = ((bc.gm[k] & 3) == 1 && dz > 0) ? 2 : bc.gm[k];
        if ((gmk & 3) == 1 || (gmk == 2 && sc.mode == 0)) continue;  // taken at conversion
        if (src == 1) {
          const double* s0 = Uin + zoff + bc.xy[k];
#pragma unroll
          for (int v = 0; v < 5; ++v) cp_async8(sStg + v * NB + p, s0 + v * d.bN);
        } else if (src == 2) {
          const float* s0 = WhS + pz + bc.pxy[k];
#pragma unroll
          for (int c = 0; c < 7; ++c) cp_async4(sStgF + 2 * ((c >> 1) * NB + p) + (c & 1), s0 + (long long)c * P);
        }
      }
      cp_async_commit();
    };

    issue(z0 - HB);
    for (int L = z0 - HB; L < z1 + HB; ++L) {
      // ---- staged plane L -> primitives in the rings (bounded wait on the bulk rows: a wait that
      // gives up records it in the status word and ends the CTA after its copies have landed)
      cp_async_wait_all();
      const bool stg_ok = mbar_wait_bounded(&sBar, stg_phase, STG_WAIT_LIMIT);
      stg_phase ^= 1u;
      if (__syncthreads_or(!stg_ok)) {
        if (tid == 0 && sc.status) atomicOr(sc.status, 1);
        mbar_wait_bounded(&sBar, stg_phase ^ 1u, STG_WAIT_LIMIT);
        return;
      }
      {
        float4* r4 = sR4 + ((L + 15) % 5) * NB;
        float4* r3 = sR3 + ((L + 15) % 3) * NW;
        const int dz = L < 0 ? -L : (L >= d.sz ? L - d.sz + 1 : 0);
#pragma unroll
        for (int k = 0; k < KB; ++k) {
          if (bc.dxy[k] < 0) continue;
          const int src = box_source(sc.mode, g.r, bc.dxy[k] & 255, bc.dxy[k] >> 8, dz);
          if (src == 0) continue;
          const int p = bc.pq[k] & 0xffff, qw = bc.pq[k] >> 16;
          float w[7];
          const int gmk = ((bc.gm[k] & 3) == 1 && dz > 0) ? 2 : bc.gm[k];  // (as in the staging)
          if ((gmk & 3) == 1) {
            // wall mirror / outflow copy: the own source point staged in this plane
            const int ps = (gmk >> 2) & 0xffff;
            const double sg = (gmk >> 18) & 1 ? -1.0 : 1.0;
            double u[5];
#pragma unroll
            for (int v = 0; v < 5; ++v) u[v] = (v >= 1 && v <= 3) ? sg * sStg[v * NB + ps] : sStg[v * NB + ps];
            prims32(u, k32, w);
          } else if (gmk == 2 && sc.mode == 0) {
            // synchronous step beyond an interface / far field: the entry's sources from the live
            // stage input, weighted (spanwise interpolation), plus the far-field constant
            const int lxc = tx0 - HB + p % BX, lyc = ty0 - HB + p / BX;
            const int gzc = wrapc(d.oz + L, d.bnz);
            const GatherEntry& E =
                g.gent[g.emap[d.ebase + (d.ox + lxc + g.GE) + (long long)d.gmx * ((d.oy + lyc + g.GE) + (long long)d.gmy * gzc)]];
            double u[5];
#pragma unroll
            for (int v = 0; v < 5; ++v) u[v] = E.cst[v];
            for (int q = 0; q < E.nt; ++q) {
              const double wt = E.w[q], wf = (E.flags[q] & 1) ? -wt : wt;
#pragma unroll
              for (int v = 0; v < 5; ++v) u[v] = fma((v >= 1 && v <= 3) ? wf : wt, Uin[E.off[q] + (long long)v * E.bN[q]], u[v]);
            }
            prims32(u, k32, w);
          } else if (src == 1) {
            double u[5];
#pragma unroll
            for (int v = 0; v < 5; ++v) u[v] = sStg[v * NB + p];
            prims32(u, k32, w);
          } else {
            const float2* s2 = reinterpret_cast<const float2*>(sStgF);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              const float2 t = s2[c * NB + p];
              w[2 * c] = t.x;
              w[2 * c + 1] = t.y;
            }
            w[6] = sStgF[2 * (3 * NB + p)];
          }
          r4[p] = make_float4(w[1], w[2], w[3], w[5]);
          if (qw != 0xffff) r3[qw] = make_float4(w[0], w[4], w[6], 0.f);
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
      const float4* pl[5];
#pragma unroll
      for (int o = 0; o < 5; ++o) pl[o] = sR4 + ((G - 2 + o + 15) % 5) * NB;  // planes G-2..G+2
      const float4* r3c = sR3 + ((G + 15) % 3) * NW;
      const bool strips = (G >= z0 && G < z1);
      float2 fz01 = make_float2(0.f, 0.f), fz23 = make_float2(0.f, 0.f);
      float fz4 = 0.f;
      // one gradient/flux evaluation at box point (bi, bj) of plane G: kind 0 tile point (Phi_x,
      // Phi_y to shared memory, Phi_z to registers), 1 x-strip (Phi_x), 2 y-strip (Phi_y)
      // Curvilinear flux point (App. A, Eq. A1-A4): the index-space gradients g0, g1 are mapped to
      // physical ones through the metric terms, d/dx_j = J sum_k (metric row k)_j d/dxi_k, and the
      // combined flux along index direction a uses the metric row m_a = (d xi_a / dx) / J:
      //   Phi_a = -[rho U, rho u U + m_a,x p, rho v U + m_a,y p, rho w U + m_a,z p, (rho E + p) U]
      //           + (1/Re) [0, m_a . tau_1, m_a . tau_2, m_a . tau_3, m_a . b],  U = m_a . u.
      // Rows: xi = (m0, m1, 0), eta = (m2, m3, 0), zeta = (0, 0, m4).
      auto curvilinear_point = [&](const float* mw, int nw, const float2* g0, const float2* g1, float4 c0, float4 c3,
                                   const Phys32& k, int kind, int bi, int bj) {
        const float m0 = mw[0], m1 = mw[nw], m2 = mw[2 * nw], m3 = mw[3 * nw], m4 = mw[4 * nw], J = mw[5 * nw];
        // physical gradients of (u, v) and (w, T) along x, y, z
        const float2 ax0 = __fmul2_rn(bc2(J), __ffma2_rn(bc2(m0), g0[0], __fmul2_rn(bc2(m2), g0[1])));
        const float2 ay0 = __fmul2_rn(bc2(J), __ffma2_rn(bc2(m1), g0[0], __fmul2_rn(bc2(m3), g0[1])));
        const float2 az0 = __fmul2_rn(bc2(J * m4), g0[2]);
        const float2 ax1 = __fmul2_rn(bc2(J), __ffma2_rn(bc2(m0), g1[0], __fmul2_rn(bc2(m2), g1[1])));
        const float2 ay1 = __fmul2_rn(bc2(J), __ffma2_rn(bc2(m1), g1[0], __fmul2_rn(bc2(m3), g1[1])));
        const float2 az1 = __fmul2_rn(bc2(J * m4), g1[2]);
        const float du[3][3] = {{ax0.x, ay0.x, az0.x}, {ax0.y, ay0.y, az0.y}, {ax1.x, ay1.x, az1.x}};
        const float dT[3] = {ax1.y, ay1.y, az1.y};
        const float u = c0.x, v = c0.y, w = c0.z, T = c0.w;
        const float rho = c3.x, p = c3.y, etH = c3.z + k.Href;
        float mu = 1.f;
        if (k.law == 1) mu = __powf(T, k.vexp);  // the hardware log2 / exp2 pair: a few ulp, FP32-form accuracy
        const float div = (du[0][0] + du[1][1]) + du[2][2];
        const float vel[3] = {u, v, w};
        float tau[3][3], bq[3];
#pragma unroll
        for (int i2 = 0; i2 < 3; ++i2)
#pragma unroll
          for (int j2 = 0; j2 < 3; ++j2)
            tau[i2][j2] = fmaf(i2 == j2 ? (-2.f / 3.f) * mu : 0.f, div, mu * (du[i2][j2] + du[j2][i2]));
#pragma unroll
        for (int i2 = 0; i2 < 3; ++i2) bq[i2] = fmaf(u, tau[i2][0], fmaf(v, tau[i2][1], fmaf(w, tau[i2][2], k.kap * mu * dT[i2])));
        const float mr[3][3] = {{m0, m1, 0.f}, {m2, m3, 0.f}, {0.f, 0.f, m4}};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          if (kind == 1 && a != 0) continue;
          if (kind == 2 && a != 1) continue;
          const float Uc = fmaf(mr[a][0], u, fmaf(mr[a][1], v, mr[a][2] * w)), mflux = rho * Uc;
          float f[5];
          f[0] = -mflux;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const float vis = fmaf(mr[a][0], tau[0][c], fmaf(mr[a][1], tau[1][c], mr[a][2] * tau[2][c]));
            f[1 + c] = fmaf(k.ire, vis, -fmaf(mflux, vel[c], mr[a][c] * p));
          }
          f[4] = fmaf(k.ire, fmaf(mr[a][0], bq[0], fmaf(mr[a][1], bq[1], mr[a][2] * bq[2])), -(etH * Uc));
          if (a == 0) {
            const int o = (bj - HB) * FXW + (bi - HB + 2);
            sFx4[o] = make_float4(f[0], f[1], f[2], f[3]);
            sFx1[o] = f[4];
          } else if (a == 1) {
            const int o = (bj - HB + 2) * FX + (bi - HB);
            sFy4[o] = make_float4(f[0], f[1], f[2], f[3]);
            sFy1[o] = f[4];
          } else {
            fz01 = make_float2(f[0], f[1]);
            fz23 = make_float2(f[2], f[3]);
            fz4 = f[4];
          }
        }
      };
      auto point = [&](int bi, int bj, int kind) {
        const float4* P0 = pl[2];
        const int q = bj * BX + bi;
        const int qw = (bj - (HB - 2)) * WX + (bi - (HB - 2));
        float2 g0[3], g1[3];  // per axis: (du, dv), (dw, dT)
        cd4_pair(P0[q - 2], P0[q - 1], P0[q + 1], P0[q + 2], c1x, c2x, g0[0], g1[0]);
        cd4_pair(P0[q - 2 * BX], P0[q - BX], P0[q + BX], P0[q + 2 * BX], c1y, c2y, g0[1], g1[1]);
        cd4_pair(pl[0][q], pl[1][q], pl[3][q], pl[4][q], c1z, c2z, g0[2], g1[2]);
        if (curv) {
          curvilinear_point(sMet + qw, NW, g0, g1, P0[q], r3c[qw], k32, kind, bi, bj);
          return;
        }
        // du[i][j] = d u_i / d x_j
        const float du[3][3] = {{g0[0].x, g0[1].x, g0[2].x}, {g0[0].y, g0[1].y, g0[2].y}, {g1[0].x, g1[1].x, g1[2].x}};
        const float dT[3] = {g1[0].y, g1[1].y, g1[2].y};
        const float4 c0 = P0[q];
        const float4 c3 = r3c[qw];
        const float u = c0.x, v = c0.y, w = c0.z, T = c0.w;
        const float rho = c3.x, p = c3.y, etH = c3.z + k32.Href;
        float mu = 1.f;
        if (k32.law == 1) mu = __powf(T, k32.vexp);
        const float div = (du[0][0] + du[1][1]) + du[2][2];
        const float m23 = (-2.f / 3.f) * mu, kmu = k32.kap * mu;
        const float vel[3] = {u, v, w};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          if (kind == 1 && a != 0) continue;
          if (kind == 2 && a != 1) continue;
          const float ua = vel[a], mflux = rho * ua;
          float tau[3];
#pragma unroll
          for (int i2 = 0; i2 < 3; ++i2) tau[i2] = mu * (du[a][i2] + du[i2][a]);
          tau[a] = fmaf(m23, div, tau[a]);
          const float qa = fmaf(u, tau[0], fmaf(v, tau[1], fmaf(w, tau[2], kmu * dT[a])));
          const float f0 = -mflux;
          const float f1 = fmaf(k32.ire, tau[0], -fmaf(mflux, u, a == 0 ? p : 0.f));
          const float f2 = fmaf(k32.ire, tau[1], -fmaf(mflux, v, a == 1 ? p : 0.f));
          const float f3 = fmaf(k32.ire, tau[2], -fmaf(mflux, w, a == 2 ? p : 0.f));
          const float f4 = fmaf(k32.ire, qa, -(etH * ua));
          if (a == 0) {
            const int o = (bj - HB) * FXW + (bi - HB + 2);
            sFx4[o] = make_float4(f0, f1, f2, f3);
            sFx1[o] = f4;
          } else if (a == 1) {
            const int o = (bj - HB + 2) * FX + (bi - HB);
            sFy4[o] = make_float4(f0, f1, f2, f3);
            sFy1[o] = f4;
          } else {
            fz01 = make_float2(f0, f1);
            fz23 = make_float2(f2, f3);
            fz4 = f4;
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
      float2 r01 = make_float2(0.f, 0.f), r23 = make_float2(0.f, 0.f);
      float r4s = 0.f;
      if (strips) {
        const int ox = ty * FXW + tx + 2, oy = (ty + 2) * FX + tx;
        const float4 xm2 = sFx4[ox - 2], xm1 = sFx4[ox - 1], xp1 = sFx4[ox + 1], xp2 = sFx4[ox + 2];
        const float4 ym2 = sFy4[oy - 2 * FX], ym1 = sFy4[oy - FX], yp1 = sFy4[oy + FX], yp2 = sFy4[oy + 2 * FX];
        r01 = __ffma2_rn(bc2(k1x), sub2(lo2(xp1), lo2(xm1)), __fmul2_rn(bc2(k2x), sub2(lo2(xp2), lo2(xm2))));
        r01 = __ffma2_rn(bc2(k1y), sub2(lo2(yp1), lo2(ym1)), r01);
        r01 = __ffma2_rn(bc2(k2y), sub2(lo2(yp2), lo2(ym2)), r01);
        r23 = __ffma2_rn(bc2(k1x), sub2(hi2(xp1), hi2(xm1)), __fmul2_rn(bc2(k2x), sub2(hi2(xp2), hi2(xm2))));
        r23 = __ffma2_rn(bc2(k1y), sub2(hi2(yp1), hi2(ym1)), r23);
        r23 = __ffma2_rn(bc2(k2y), sub2(hi2(yp2), hi2(ym2)), r23);
        r4s = fmaf(k1x, sFx1[ox + 1] - sFx1[ox - 1], k2x * (sFx1[ox + 2] - sFx1[ox - 2]));
        r4s = fmaf(k1y, sFy1[oy + FX] - sFy1[oy - FX], r4s);
        r4s = fmaf(k2y, sFy1[oy + 2 * FX] - sFy1[oy - 2 * FX], r4s);
      }
      float out[5];
      {
        const float2 o01 = __ffma2_rn(bc2(k2z), fz01, aq[0][0]), o23 = __ffma2_rn(bc2(k2z), fz23, aq[0][1]);
        aq[0][0] = __ffma2_rn(bc2(k1z), fz01, aq[1][0]);
        aq[0][1] = __ffma2_rn(bc2(k1z), fz23, aq[1][1]);
        aq[1][0] = __fadd2_rn(aq[2][0], r01);
        aq[1][1] = __fadd2_rn(aq[2][1], r23);
        aq[2][0] = __ffma2_rn(bc2(-k1z), fz01, aq[3][0]);
        aq[2][1] = __ffma2_rn(bc2(-k1z), fz23, aq[3][1]);
        aq[3][0] = __fmul2_rn(bc2(-k2z), fz01);
        aq[3][1] = __fmul2_rn(bc2(-k2z), fz23);
        out[0] = o01.x;
        out[1] = o01.y;
        out[2] = o23.x;
        out[3] = o23.y;
        out[4] = fmaf(k2z, fz4, aq4[0]);
        aq4[0] = fmaf(k1z, fz4, aq4[1]);
        aq4[1] = aq4[2] + r4s;
        aq4[2] = fmaf(-k1z, fz4, aq4[3]);
        aq4[3] = -k2z * fz4;
      }
      if (outp) {
        // no-slip wall points keep zero momentum (connected grids)
        const bool wallpt = d.wall && ((((d.wall >> 0) & 1) && lx == 0) || (((d.wall >> 1) & 1) && lx == d.sx - 1) ||
                                       (((d.wall >> 2) & 1) && ly == 0) || (((d.wall >> 3) & 1) && ly == d.sy - 1));
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          const double dtR = curv ? f2d_fast(out[c]) * Jown : f2d_fast(out[c]);  // index-space divergence x J
          double qn = first ? dtR : fma(A, qin[c], dtR);
          double un = fma(B, qn, uin[c]);
          if (wallpt && c >= 1 && c <= 3) qn = un = 0.0;
          if (!last) Q[c * d.bN + go] = qn;
          Uout[c * d.bN + go] = un;
        }
      }
    }
  }
}

// ------------------------------------------------------------------------------- launchers

int fused_smem_bytes(int fy, int curv) {
  if (fy == 4) return (int)(curv ? FusedSmem<32, 4>::bytes_curv : FusedSmem<32, 4>::bytes);
  if (fy == 16) return (int)(curv ? FusedSmem<32, 16>::bytes_curv : FusedSmem<32, 16>::bytes);
  return (int)(curv ? FusedSmem<32, 8>::bytes_curv : FusedSmem<32, 8>::bytes);
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
static int fused_prepare(int* blocks_per_sm, int curv) {
  const size_t sm = curv ? FusedSmem<FX, FY>::bytes_curv : FusedSmem<FX, FY>::bytes;
  // the shared-memory opt-in (the largest size) is a per-device attribute of the kernel
  static std::mutex mu;
  static bool attr_set[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return (int)e;
  if (dev < 0 || dev >= 64) return (int)cudaErrorInvalidDevice;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!attr_set[dev]) {
      e = cudaFuncSetAttribute(k_stage_fused<FX, FY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)FusedSmem<FX, FY>::bytes_curv);
      if (e != cudaSuccess) return (int)e;
      attr_set[dev] = true;
    }
  }
  if (blocks_per_sm) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_stage_fused<FX, FY>, FX * FY, sm);
    if (e != cudaSuccess) return (int)e;
  }
  return 0;
}

int fused_blocks_per_sm(int fy, int curv, int* blocks) {
  if (fy == 4) return fused_prepare<32, 4>(blocks, curv);
  if (fy == 16) return fused_prepare<32, 16>(blocks, curv);
  return fused_prepare<32, 8>(blocks, curv);
}

template <int FX, int FY>
static int fused_impl(const Geometry& g, const Physics& ph, const StepSched& sc, const FusedLaunch& a, cudaStream_t st) {
  const int rc = fused_prepare<FX, FY>(nullptr, a.curv);
  if (rc) return rc;
  k_stage_fused<FX, FY><<<a.grid, FX * FY, a.curv ? FusedSmem<FX, FY>::bytes_curv : FusedSmem<FX, FY>::bytes, st>>>(
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
