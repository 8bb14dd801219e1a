// kernels.cu -- CUDA kernels (sm_103a) of the asynchronous compressible-flow hot path.
//
// One LSERK stage (Eq. 3) of the method of arXiv 2506.03027 runs as three kernels over every
// sub-domain ("PE", Sec. 3):
//   k_view  : the stage input U^(m-1) as the sub-domain sees it -- its own points plus a halo
//             taken from the live neighbour values (SA, Alg. 1), from the delayed levels of the
//             ring combined with the AT weights W^(m-1)(k) (Eq. 14-15 at m = 1, then the buffer
//             updates of Eq. 8 / Table 5 collapsed into weights), or from the latest delayed level
//             (AS) -- converted to primitives (App. A).
//   k_flux  : combined fluxes Phi_a = -F_a + Fv_a / Re (Eq. A2-A4) at the owned points and at
//             the halo points within the stencil radius along a; viscous gradients by CD.
//   k_rk    : R = sum_a D_a Phi_a with the CD scheme of Eq. 2, fused with the low-storage RK
//             update Q = A Q + dt R, U^(m) = U^(m-1) + B Q (FP64 accumulation).
// The tenth-order Pade filter (once per step) is k_filter, one tridiagonal line solve per
// thread with a Dirichlet closure at the first halo point.  k_diag* reduce the diagnostics.
//
// Data layout: global state arrays are SoA FP64 [5][nz][ny][nx]; the ring holds R full states
// (level t in slot t mod R).  Scratch arrays are component-major over the concatenated padded
// boxes of all sub-domains.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <type_traits>
#include <utility>

#include "cfs_internal.h"
#include "device_common.cuh"

namespace cfs {

// Programmatic dependent launch: the kernels of the FP64 stage sequence (view, flux, stage update,
// filter passes, step counter) are launched with programmatic stream serialization, so the next
// kernel's CTAs are scheduled while this one drains.  Every such kernel first lets its successor
// launch, then waits for its predecessor to complete (and its memory to be visible) before it
// reads anything the predecessor wrote; launched without the attribute both are no-ops.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
}

template <typename... KArgs, typename... Args>
static inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// ------------------------------------------------------------------------------- k_view

// Store the primitives of conserved state u at padded index q of sub-domain d (App. A:
// p = (gamma-1)(rho E - rho|u|^2/2), T = gamma M^2 p / rho).  In the FP32 form p and rho E are
// carried as deviations from p_ref and E_ref (exact algebra: the constant part of p has no
// derivative and the constant enthalpy H_ref is added back in k_flux).
template <typename T>
__device__ __forceinline__ void store_prims(const Geometry& g, const Physics& ph, const double* u, long long o,
                                            T* __restrict__ Wp) {
  constexpr bool f32 = std::is_same<T, float>::value;
  const T rho = (T)u[0];
  const T ir = recip(rho);
  const T uu = (T)u[1] * ir, vv = (T)u[2] * ir, ww = (T)u[3] * ir;
  const T ke = (T)0.5 * ((T)u[1] * uu + (T)u[2] * vv + (T)u[3] * ww);
  const T rE = f32 ? (T)(u[4] - ph.E_ref) : (T)u[4];
  const T p = (T)ph.gm1 * (rE - ke);
  // kappa T (the heat flux kappa mu dT/dx is then mu times its gradient)
  const T temp = f32 ? fma((T)ph.kgM2, p, (T)ph.kappa) * ir : (T)ph.kgM2 * p * ir;
  const long long P = g.Ptot;
  Wp[o] = rho;
  Wp[P + o] = uu;
  Wp[2 * P + o] = vv;
  Wp[3 * P + o] = ww;
  Wp[4 * P + o] = p;
  Wp[5 * P + o] = temp;
  Wp[6 * P + o] = rE + p;  // rho E + p (energy flux factor; minus H_ref in the FP32 form)
}

// k_view, owned points: the stage input of the sub-domain's own points as primitives (thread t
// of sub-domain sid).
template <typename T>
__device__ __forceinline__ void view_own(const Geometry& g, const Physics& ph, const double* __restrict__ Uin,
                                         const SubDev* __restrict__ subs, T* __restrict__ Wp, int sid, int t) {
  const SubDev d = subs[sid];
  if (!d.own) return;  // another process's sub-domain
  if (t >= d.sx * d.sy * d.sz) return;
  const int sxy = d.sx * d.sy, ck = t / sxy, r2 = t - ck * sxy, cj = r2 / d.sx, ci = r2 - cj * d.sx;
  const long long gi = (long long)(d.ox + ci) + (long long)d.bnx * ((long long)(d.oy + cj) + (long long)d.bny * (d.oz + ck));
  const long long q = (long long)(ci + g.G) + (long long)d.ex * ((long long)(cj + g.G) + (long long)d.ey * (ck + g.Gz));
  double u[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) u[v] = Uin[d.bbase + v * d.bN + gi];
  store_prims<T>(g, ph, u, d.pbase + q, Wp);
}

// k_view, halo points: one thread per entry of the compact list of (sub-domain, padded index) of
// the points a sub-domain reads from neighbours -- faces to depth G, viscous edges to r x r -- so
// that no warp mixes owned points with the AT weighting.  SA: the neighbour's live value; AT:
// sum_l W^(m)_l(k) U^{n-k-l} in FP64 (Eq. 14-15, buffer updates of Eq. 8 collapsed); AS: U^{n-k}.
template <typename T>
__device__ __forceinline__ void view_halo(const Geometry& g, const Physics& ph, const StepSched& sc,
                                          const double* __restrict__ Uin, const double* __restrict__ ring,
                                          const SubDev* __restrict__ subs, const int2* __restrict__ halo, long long nhalo,
                                          T* __restrict__ Wp, int stage, int s, long long t) {
  if (t >= nhalo) return;
  const int2 e = halo[t];
  const int sid = e.x;
  const int q = e.y;  // index in the sub-domain's padded box (32-bit)
  const SubDev d = subs[sid];
  const int exy = d.ex * d.ey;
  const int k = q / exy, r2 = q - k * exy, j = r2 / d.ex, i = r2 - j * d.ex;
  const int ci = i - g.G, cj = j - g.G, ck = k - g.Gz;
  // halo points lie within G of the sub-domain: one conditional wrap per axis
  auto wrap1 = [](int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); };
  const int gx = wrap1(d.ox + ci, d.bnx), gy = wrap1(d.oy + cj, d.bny), gz = wrap1(d.oz + ck, d.bnz);
  const long long gi = d.bbase + (long long)gx + (long long)d.bnx * ((long long)gy + (long long)d.bny * gz);
  // ring slot of level n - kd - l: (n mod R) - kd - l, wrapped once (kd + l < R)
  const int nR = (int)(sc.n % sc.R);
  double u[5];
  const int ux = d.ox + ci, uy = d.oy + cj;
  if (d.ebase >= 0 && (ux < 0 || ux >= d.bnx || uy < 0 || uy >= d.bny)) {
    // beyond a non-periodic block face: own sources (wall mirror, outflow copy) current, a
    // neighbouring PE's by the mode with the delay of the faces crossed (physical faces carry
    // none), far-field constants
    int kd = 0;
    if (sc.mode != 0) {
      if ((ci < 0 || ci >= d.sx) && !((d.phys >> (ci < 0 ? 0 : 1)) & 1)) kd = max(kd, face_delay(sc, sid, ci < 0 ? 0 : 1));
      if ((cj < 0 || cj >= d.sy) && !((d.phys >> (cj < 0 ? 2 : 3)) & 1)) kd = max(kd, face_delay(sc, sid, cj < 0 ? 2 : 3));
      if ((ck < 0 || ck >= d.sz) && !((d.phys >> (ck < 0 ? 4 : 5)) & 1)) kd = max(kd, face_delay(sc, sid, ck < 0 ? 4 : 5));
    }
    auto slot = [&](int l) { const int qq = nR - kd - l; return qq < 0 ? qq + sc.R : qq; };
    const bool zin = ck >= 0 && ck < d.sz;
    const int ei = g.emap[d.ebase + (ux + g.GE) + (long long)d.gmx * ((uy + g.GE) + (long long)d.gmy * gz)];
    const GatherEntry& E = g.gent[ei];
#pragma unroll
    for (int v = 0; v < 5; ++v) u[v] = E.cst[v];
    const long long lvN = 5 * g.N;
    const double* w = sc.W + (kd * s + stage) * sc.C;
    for (int t = 0; t < E.nt; ++t) {
      // an own source (wall mirror, outflow copy of this sub-domain's point) is current only for
      // points inside the sub-domain in z: the map is indexed at the wrapped z, so beyond a z
      // face the source is reached across the periodic wrap -- a neighbouring PE's in z (with a
      // single sub-domain along z, the sub-domain's own PE across that face), seen with delay
      const bool own = zin && !(E.flags[t] & 2) && E.sid[t] == sid;
      const double wt = E.w[t], wf = (E.flags[t] & 1) ? -wt : wt;
      const long long o = E.off[t];
      const long long bN = E.bN[t];
      double x[5];
      if (own || sc.mode == 0) {
#pragma unroll
        for (int v = 0; v < 5; ++v) x[v] = Uin[o + v * bN];
      } else if (sc.mode == 2) {
        const double* src = ring + (long long)slot(0) * lvN;
#pragma unroll
        for (int v = 0; v < 5; ++v) x[v] = src[o + v * bN];
      } else {
#pragma unroll
        for (int v = 0; v < 5; ++v) x[v] = 0.0;
        for (int l = 0; l < sc.C; ++l) {
          const double* src = ring + (long long)slot(l) * lvN;
          const double wl = __ldg(w + l);
#pragma unroll
          for (int v = 0; v < 5; ++v) x[v] = fma(wl, src[o + v * bN], x[v]);
        }
      }
#pragma unroll
      for (int v = 0; v < 5; ++v) u[v] = fma((v >= 1 && v <= 3) ? wf : wt, x[v], u[v]);
    }
    store_prims<T>(g, ph, u, d.pbase + q, Wp);
    return;
  }
  if (sc.mode == 0) {
#pragma unroll
    for (int v = 0; v < 5; ++v) u[v] = Uin[v * d.bN + gi];
  } else {
    int kd = 0;  // (faces inside the block: none is physical)
    if (ci < 0 || ci >= d.sx) kd = max(kd, face_delay(sc, sid, ci < 0 ? 0 : 1));
    if (cj < 0 || cj >= d.sy) kd = max(kd, face_delay(sc, sid, cj < 0 ? 2 : 3));
    if (ck < 0 || ck >= d.sz) kd = max(kd, face_delay(sc, sid, ck < 0 ? 4 : 5));
    const long long lvN = 5 * g.N;
    auto slot = [&](int l) { const int qq = nR - kd - l; return qq < 0 ? qq + sc.R : qq; };
    if (sc.mode == 2) {
      const double* src = ring + (long long)slot(0) * lvN;
#pragma unroll
      for (int v = 0; v < 5; ++v) u[v] = src[v * d.bN + gi];
    } else {
      const double* w = sc.W + (kd * s + stage) * sc.C;
      const bool face = (int)(ci < 0 || ci >= d.sx) + (int)(cj < 0 || cj >= d.sy) + (int)(ck < 0 || ck >= d.sz) == 1;
      if (sc.LH && face) {
        // learned stage-0 value (per face column, from the network) plus the AT buffer-update
        // increments (W^(m) - W^(0)) applied to the delayed levels
        const double* w0 = sc.W + (kd * s) * sc.C;
#pragma unroll
        for (int v = 0; v < 5; ++v) u[v] = sc.LH[(long long)v * g.Ptot + d.pbase + q];
        if (stage > 0)
          for (int l = 0; l < sc.C; ++l) {
            const double* src = ring + (long long)slot(l) * lvN;
            const double wl = __ldg(w + l) - __ldg(w0 + l);
#pragma unroll
            for (int v = 0; v < 5; ++v) u[v] = fma(wl, src[v * d.bN + gi], u[v]);
          }
      } else {
#pragma unroll
        for (int v = 0; v < 5; ++v) u[v] = 0.0;
        for (int l = 0; l < sc.C; ++l) {
          const double* src = ring + (long long)slot(l) * lvN;
          const double wl = __ldg(w + l);
#pragma unroll
          for (int v = 0; v < 5; ++v) u[v] = fma(wl, src[v * d.bN + gi], u[v]);
        }
      }
    }
  }
  store_prims<T>(g, ph, u, d.pbase + q, Wp);
}

// The stage input as primitives, own points and halo points in one launch: the first own_blocks x
// nsub CTAs take the owned points (own_blocks CTAs per sub-domain), the rest the halo list.
template <typename T>
__global__ void __launch_bounds__(512) k_view(Geometry g, Physics ph, StepSched sc, const double* __restrict__ Uin0,
                                              const double* __restrict__ ring, int in_ring, const SubDev* __restrict__ subs,
                                              const int2* __restrict__ halo, long long nhalo, T* __restrict__ Wp,
                                              int stage, int s, int own_blocks) {
  pdl_enter();
  sc = resolve(sc);
  const double* Uin = ring_or(Uin0, in_ring, ring, sc, 0);
  const long long b = blockIdx.x, nown = (long long)own_blocks * g.nsub;
  if (b < nown) {
    const int sid = (int)(b / own_blocks);
    view_own<T>(g, ph, Uin, subs, Wp, sid, (int)(b - (long long)sid * own_blocks) * blockDim.x + threadIdx.x);
  } else {
    view_halo<T>(g, ph, sc, Uin, ring, subs, halo, nhalo, Wp, stage, s, (b - nown) * blockDim.x + threadIdx.x);
  }
}

// ------------------------------------------------------------------------------- k_flux

// x^a = exp(a ln x) in FP64 for positive normal x (the viscosity law mu = T^a), table-driven
// after Tang (ACM TOMS 1989, 1990), about 20 FP64 operations.  ln x: x = m 2^e with m in [1, 2)
// from the bit fields; the top six mantissa bits pick c_j = 1 + (j + 1/2)/64, u = m / c_j - 1
// (|u| <= 1/129) from a table of 1/c_j, ln m = ln c_j + log1p(u) with the series of log1p to u^7.
// exp y: y = (64 k' + j') ln2/64 + r with |r| <= ln2/128 (ln 2 / 64 split into a 32-bit head and
// its tail: k ln2_head is exact), exp r by its Taylor series to r^5/5!, times the tabulated
// 2^(j'/64), and 2^k' added to the exponent field.  Tables: 1/c_j rounded from the exact
// quotient, ln c_j and 2^(j/64) rounded from long-double log1p and exp2 (pow_tables_init).
// Relative error below 6e-16 (1 + |a ln x|).  Any other x, or |a ln x| >= 700, goes to the
// library's pow.
__device__ double g_pow_tab[3 * 64];  // 1/c_j, ln c_j, 2^(j/64)

__device__ __forceinline__ double pow_tab(double x, double a) {
  if (!(x >= 2.2250738585072014e-308) || !(x <= 1.7976931348623157e308)) return pow(x, a);
  const int hi = __double2hiint(x);
  const int e = ((hi >> 20) & 0x7ff) - 1023;
  const int j = (hi >> 14) & 63;
  const double m = __hiloint2double((hi & 0x000fffff) | 0x3ff00000, __double2loint(x));  // [1, 2)
  const double u = fma(m, __ldg(g_pow_tab + j), -1.0);
  double p = 1.0 / 7.0;
  p = fma(p, u, -1.0 / 6.0);
  p = fma(p, u, 1.0 / 5.0);
  p = fma(p, u, -1.0 / 4.0);
  p = fma(p, u, 1.0 / 3.0);
  p = fma(p, u, -0.5);
  p = fma(p, u, 1.0);
  const double l1p = p * u;
  const double LN2_HEAD = 0.6931471803691238, LN2_TAIL = 1.9082149292705877e-10;
  const double ed = (double)e;
  // (e ln2_head + ln c_j) is exact where it cancels (x just below 1: Sterbenz), then the tails
  const double y = a * (fma(ed, LN2_HEAD, __ldg(g_pow_tab + 64 + j)) + fma(ed, LN2_TAIL, l1p));
  if (!(fabs(y) < 700.0)) return pow(x, a);
  const double kd = rint(y * (64.0 / 0.6931471805599453));
  double r = fma(-kd, LN2_HEAD / 64.0, y);
  r = fma(-kd, LN2_TAIL / 64.0, r);
  double q = 1.0 / 120.0;
  q = fma(q, r, 1.0 / 24.0);
  q = fma(q, r, 1.0 / 6.0);
  q = fma(q, r, 0.5);
  q = fma(q, r, 1.0);
  q = fma(q, r, 1.0);
  const int k = (int)kd;
  q *= __ldg(g_pow_tab + 128 + (k & 63));
  return __hiloint2double(__double2hiint(q) + ((k >> 6) << 20), __double2loint(q));
}

// Viscosity law: mu = 1, or the power law mu = T^visc_exp -- in the intermediate precision (the
// FP32 form evaluates it in FP32 with the hardware log2 / exp2 pair, a few ulp: a power in FP64
// runs at the FP64 rate).  The flux kernels pass
// kappa T and take the factor kappa^-a with 1/Re (Physics::ivT).
template <typename T>
__device__ __forceinline__ T visc_mu(const Physics& ph, T temp) {
  if (ph.visc_law != 1) return (T)1;
  if (std::is_same<T, float>::value) return (T)__powf((float)temp, (float)ph.visc_exp);
  return (T)pow_tab((double)temp, ph.visc_exp);
}

template <typename T>
__device__ __forceinline__ T cdiff(const T* __restrict__ f, long long q, long long st, T c1, T c2, int r) {
  T d = c1 * (f[q + st] - f[q - st]);
  if (r == 2) d = fma(c2, f[q + 2 * st] - f[q - 2 * st], d);
  return d;
}

// The same difference without its factor: CD4 (f_{+2} - f_{-2}) - 8 (f_{+1} - f_{-1}) (times c2
// gives cdiff), CD2 f_{+1} - f_{-1} (times c1)
template <typename T>
__device__ __forceinline__ T cdiff_iso(const T* __restrict__ f, long long q, long long st, int r) {
  const T d1 = f[q + st] - f[q - st];
  return r == 2 ? fma((T)-8, d1, f[q + 2 * st] - f[q - 2 * st]) : d1;
}

// Curvilinear flux point (App. A, Eq. A1-A4 with a time-invariant grid): gradients in index
// space, mapped to physical gradients by d phi / d x_j = J sum_k (metric row k)_j d phi / d xi_k;
// combined fluxes along each index direction a with the metric row
// m_a = (d xi_a / dx, d xi_a / dy, d xi_a / dz) / J:
//   Phi_a = -[rho U^, rho u U^ + m_x p, rho v U^ + m_y p, rho w U^ + m_z p, (rho E + p) U^]
//           + (1/Re) [0, m . tau_1, m . tau_2, m . tau_3, m . b],   U^ = m . u.
// The grid is extruded in z: rows xi = (a00, a01, 0), eta = (a10, a11, 0), zeta = (0, 0, a22), so
// the products with the zero entries are left out.  The index spacing is 1 on every axis, so the
// differences are taken without their factor gs (as cdiff_iso); the viscous flux is linear in the
// gradients, so gs, J and mu multiply it once, in iv.  A strip point evaluates the flux along its
// axis only, with the temperature gradients that flux needs.
template <typename T, int ND>
__device__ __forceinline__ void flux_curvilinear(const Geometry& g, const Physics& ph, const SubDev& d,
                                                 const T* __restrict__ W, T* __restrict__ out, long long q, int ci,
                                                 int cj, int ck, bool ox, bool oy, bool oz, int nout) {
  const long long P = g.Ptot;
  const int r = g.r;
  const long long sty = d.ex, stz = (long long)d.ex * d.ey;
  // metric plane of the block (extended by G, z-independent): flux points lie within r <= G
  const double* M = g.metric + d.mbase + (long long)(d.ox + ci + g.G) + (long long)d.mx * (d.oy + cj + g.G);
  const long long pl = d.mpl;
  const T a00 = (T)M[0], a01 = (T)M[pl], a10 = (T)M[2 * pl], a11 = (T)M[3 * pl], a22 = (T)M[4 * pl];
  const T rho = W[q], u = W[P + q], v = W[2 * P + q], w = W[3 * P + q], p = W[4 * P + q];
  const T et = W[6 * P + q];
  // tau / (gs J mu) and b / (gs J mu) (b_i = u_j tau_ij + kappa mu dT/dx_i)
  T t00 = 0, t11 = 0, t22 = 0, t01 = 0, t02 = 0, t12 = 0, b0 = 0, b1 = 0, b2 = 0;
  T iv = (T)ph.ivT;
  if (g.viscous) {
    const long long st[3] = {1, sty, stz};
    const bool needTxy = nout == 0 || !oz, needTz = nout == 0 || oz;
    T dxi[4][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {0, 0, 0}};  // d (u, v, w, T) / d xi_k / gs
#pragma unroll
    for (int k = 0; k < ND; ++k) {
#pragma unroll
      for (int c = 0; c < 3; ++c) dxi[c][k] = cdiff_iso(W + (1 + c) * P, q, st[k], r);
      if (k < 2 ? needTxy : needTz) dxi[3][k] = cdiff_iso(W + 5 * P, q, st[k], r);
    }
    T G[4][3];  // physical gradients / (gs J)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      G[c][0] = fma(a10, dxi[c][1], a00 * dxi[c][0]);
      G[c][1] = fma(a11, dxi[c][1], a01 * dxi[c][0]);
      G[c][2] = ND == 3 ? a22 * dxi[c][2] : (T)0;
    }
    const T d23 = (T)(-2.0 / 3.0) * (G[0][0] + G[1][1] + G[2][2]);
    t00 = fma((T)2, G[0][0], d23);
    t11 = fma((T)2, G[1][1], d23);
    t22 = fma((T)2, G[2][2], d23);
    t01 = G[0][1] + G[1][0];
    t02 = G[0][2] + G[2][0];
    t12 = G[1][2] + G[2][1];
    // the temperature slot holds kappa T: G[3] is the heat-flux gradient
    b0 = fma(u, t00, fma(v, t01, fma(w, t02, G[3][0])));
    b1 = fma(u, t01, fma(v, t11, fma(w, t12, G[3][1])));
    b2 = fma(u, t02, fma(v, t12, fma(w, t22, G[3][2])));
    iv *= (T)(r == 2 ? d.c2[0] : d.c1[0]) * (T)M[6 * pl];
    if (ph.visc_law == 1) iv *= visc_mu<T>(ph, W[5 * P + q]);
  }
#pragma unroll
  for (int a = 0; a < ND; ++a) {
    if (nout == 1) {
      if ((a == 0 && !ox) || (a == 1 && !oy) || (a == 2 && !oz)) continue;
    }
    T f[5];
    if (a < 2) {
      const T m0 = a == 0 ? a00 : a10, m1 = a == 0 ? a01 : a11;
      const T Uc = fma(m1, v, m0 * u);
      const T nm = -rho * Uc;
      f[0] = nm;
      f[1] = fma(nm, u, -(m0 * p));
      f[2] = fma(nm, v, -(m1 * p));
      f[3] = nm * w;
      f[4] = std::is_same<T, float>::value ? -(et * Uc + (T)ph.H_ref * Uc) : -et * Uc;
      if (g.viscous) {
        f[1] = fma(iv, fma(m1, t01, m0 * t00), f[1]);
        f[2] = fma(iv, fma(m1, t11, m0 * t01), f[2]);
        f[3] = fma(iv, fma(m1, t12, m0 * t02), f[3]);
        f[4] = fma(iv, fma(m1, b1, m0 * b0), f[4]);
      }
    } else {
      const T Uc = a22 * w;
      const T nm = -rho * Uc;
      f[0] = nm;
      f[1] = nm * u;
      f[2] = nm * v;
      f[3] = fma(nm, w, -(a22 * p));
      f[4] = std::is_same<T, float>::value ? -(et * Uc + (T)ph.H_ref * Uc) : -et * Uc;
      if (g.viscous) {
        const T iz = iv * a22;
        f[1] = fma(iz, t02, f[1]);
        f[2] = fma(iz, t12, f[2]);
        f[3] = fma(iz, t22, f[3]);
        f[4] = fma(iz, b2, f[4]);
      }
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) out[(long long)(a * 5 + c) * P + q] = f[c];
  }
}

// Flux points of a sub-domain, in warp-uniform groups: first the owned points (x fastest), then
// the strips of 2r points beyond each face where only the flux along that axis is needed (x
// strips: the 2r columns fastest, then y and z; y strips: x fastest; z strips: x fastest).  A warp
// of strip points evaluates one flux direction and only the gradients it needs.
template <int ND>
__device__ __forceinline__ bool flux_point(const SubDev& d, int r, int t, int& ci, int& cj, int& ck, int& kind) {
  const int sxy = d.sx * d.sy, nown = sxy * d.sz;
  if (t < nown) {
    ck = t / sxy;
    const int r2 = t - ck * sxy;
    cj = r2 / d.sx;
    ci = r2 - cj * d.sx;
    kind = 0;
    return true;
  }
  t -= nown;
  const int w = 2 * r;
  const int nx = w * d.sy * d.sz;
  if (t < nx) {  // x strips
    const int s = t % w, rest = t / w;
    cj = rest % d.sy;
    ck = rest / d.sy;
    ci = s < r ? s - r : d.sx + s - r;
    kind = 1;
    return true;
  }
  t -= nx;
  const int ny = w * d.sx * d.sz;
  if (t < ny) {  // y strips
    ci = t % d.sx;
    const int rest = t / d.sx, s = rest % w;
    ck = rest / w;
    cj = s < r ? s - r : d.sy + s - r;
    kind = 2;
    return true;
  }
  t -= ny;
  if (ND == 3 && t < w * sxy) {  // z strips
    ci = t % d.sx;
    const int rest = t / d.sx;
    cj = rest % d.sy;
    const int s = rest / d.sy;
    ck = s < r ? s - r : d.sz + s - r;
    kind = 3;
    return true;
  }
  return false;
}

// CURV: the context has curvilinear blocks (their flux points take flux_curvilinear), so the
// Cartesian instantiation keeps a register allocation of its own.
template <typename T, int ND, bool CURV>
__global__ void __launch_bounds__(512) k_flux(Geometry g, Physics ph, const SubDev* __restrict__ subs,
                                                            const T* __restrict__ Wp, T* __restrict__ Phi) {
  pdl_enter();
  const int sid = blockIdx.y;
  const SubDev d = subs[sid];
  if (!d.own) return;  // another process's sub-domain
  const int r = g.r;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;  // flux points of a sub-domain: < 2^31
  int ci, cj, ck, kind;
  if (!flux_point<ND>(d, g.fs, t, ci, cj, ck, kind)) return;
  const bool ox = kind == 1, oy = kind == 2, oz = kind == 3;
  const int nout = kind > 0 ? 1 : 0;
  const long long sty = d.ex, stz = (long long)d.ex * d.ey;
  const long long q = (long long)(ci + g.G) + sty * (cj + g.G) + stz * (ck + g.Gz);
  const long long P = g.Ptot;
  const T* W = Wp + d.pbase;
  if (CURV && d.mbase >= 0) {
    flux_curvilinear<T, ND>(g, ph, d, W, Phi + d.pbase, q, ci, cj, ck, ox, oy, oz, nout);
    return;
  }
  const T rho = W[q], u = W[P + q], v = W[2 * P + q], w = W[3 * P + q], p = W[4 * P + q];
  const T et = W[6 * P + q];
  const T vel[3] = {u, v, w};
  // gradients du[i][j] = d u_i / d x_j, dT[j].  A strip point beyond the faces of axis a needs the
  // flux along a only: du[a][*], du[*][a], du[b][b] (the divergence) and dT[a].  With the same
  // spacing on every axis they are taken in units of the common factor gs (CD4: a = 4/3, b = -1/3
  // make c1 = -8 c2, so d = c2 ((f_{+2} - f_{-2}) - 8 (f_{+1} - f_{-1})); CD2: d = c1 (f_{+1} -
  // f_{-1})): the viscous flux is linear in them, so gs joins 1/Re (and mu) in one factor.
  T du[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  T dT[3] = {0, 0, 0};
  T iv = (T)ph.ivT;  // the factor of the viscous terms: 1/Re x gs x mu
  const int as = kind - 1;  // strip axis (-1: owned point)
  if (g.viscous) {
    const long long st[3] = {1, sty, stz};
    // (compared as bit patterns: an FP64 compare would occupy the FP64 pipe)
    bool iso = true;
#pragma unroll
    for (int b = 1; b < ND; ++b)
      iso = iso && __double_as_longlong(d.c1[b]) == __double_as_longlong(d.c1[0]) &&
            __double_as_longlong(d.c2[b]) == __double_as_longlong(d.c2[0]);
    if (iso) {
#pragma unroll
      for (int b = 0; b < ND; ++b) {
        const bool all = as < 0 || as == b;
        if (all || as == 0 || b == 0) du[0][b] = cdiff_iso(W + P, q, st[b], r);
        if (all || as == 1 || b == 1) du[1][b] = cdiff_iso(W + 2 * P, q, st[b], r);
        if (all || as == 2 || b == 2) du[2][b] = cdiff_iso(W + 3 * P, q, st[b], r);
        if (all) dT[b] = cdiff_iso(W + 5 * P, q, st[b], r);
      }
      iv *= (T)(r == 2 ? d.c2[0] : d.c1[0]);
    } else {
#pragma unroll
      for (int b = 0; b < ND; ++b) {
        const T c1 = (T)d.c1[b], c2 = (T)d.c2[b];
        const bool all = as < 0 || as == b;
        if (all || as == 0 || b == 0) du[0][b] = cdiff(W + P, q, st[b], c1, c2, r);
        if (all || as == 1 || b == 1) du[1][b] = cdiff(W + 2 * P, q, st[b], c1, c2, r);
        if (all || as == 2 || b == 2) du[2][b] = cdiff(W + 3 * P, q, st[b], c1, c2, r);
        if (all) dT[b] = cdiff(W + 5 * P, q, st[b], c1, c2, r);
      }
    }
    if (ph.visc_law == 1) iv *= visc_mu<T>(ph, W[5 * P + q]);
  }
  // tau_ai = mu (du_a/dx_i + du_i/dx_a - 2/3 div delta_ai), q_a = u_i tau_ai + kappa mu dT/dx_a:
  // mu is in iv; the symmetric sums are shared by the axes
  const T d23 = (T)(-2.0 / 3.0) * (du[0][0] + du[1][1] + du[2][2]);
  const T s01 = du[0][1] + du[1][0], s02 = du[0][2] + du[2][0], s12 = du[1][2] + du[2][1];
  T* out = Phi + d.pbase;
  constexpr bool F32 = std::is_same<T, float>::value;
  if (nout == 0) {
    // owned point, every axis: the momentum flux -rho u_a u_c - p delta_ac + tau_ac / Re is
    // symmetric in (a, c), so its six distinct entries are formed once
    const T n0 = -rho * u, n1 = -rho * v, n2 = -rho * w;  // -rho u_a
    T m00 = fma(n0, u, -p), m11 = fma(n1, v, -p), m22 = fma(n2, w, -p);
    T m01 = n0 * v, m02 = n0 * w, m12 = n1 * w;
    T e0 = F32 ? -(et * u + (T)ph.H_ref * u) : -et * u;
    T e1 = F32 ? -(et * v + (T)ph.H_ref * v) : -et * v;
    T e2 = F32 ? -(et * w + (T)ph.H_ref * w) : -et * w;
    if (g.viscous) {
      const T t00 = fma((T)2, du[0][0], d23), t11 = fma((T)2, du[1][1], d23), t22 = fma((T)2, du[2][2], d23);
      m00 = fma(iv, t00, m00);
      m11 = fma(iv, t11, m11);
      m22 = fma(iv, t22, m22);
      m01 = fma(iv, s01, m01);
      m02 = fma(iv, s02, m02);
      m12 = fma(iv, s12, m12);
      e0 = fma(iv, fma(u, t00, fma(v, s01, fma(w, s02, dT[0]))), e0);
      e1 = fma(iv, fma(u, s01, fma(v, t11, fma(w, s12, dT[1]))), e1);
      e2 = fma(iv, fma(u, s02, fma(v, s12, fma(w, t22, dT[2]))), e2);
    }
    const T f[3][5] = {{n0, m00, m01, m02, e0}, {n1, m01, m11, m12, e1}, {n2, m02, m12, m22, e2}};
#pragma unroll
    for (int a = 0; a < ND; ++a)
#pragma unroll
      for (int c = 0; c < 5; ++c) out[(long long)(a * 5 + c) * P + q] = f[a][c];
    return;
  }
  // strip point: the flux along its axis only
#pragma unroll
  for (int a = 0; a < ND; ++a) {
    if ((a == 0 && !ox) || (a == 1 && !oy) || (a == 2 && !oz)) continue;
    const T ua = vel[a];
    const T nm = -rho * ua;  // -rho u_a
    T f[5];
    f[0] = nm;
    f[1] = a == 0 ? fma(nm, u, -p) : nm * u;
    f[2] = a == 1 ? fma(nm, v, -p) : nm * v;
    f[3] = a == 2 ? fma(nm, w, -p) : nm * w;
    f[4] = F32 ? -(et * ua + (T)ph.H_ref * ua) : -et * ua;
    if (g.viscous) {
      T tau[3];
      tau[0] = a == 0 ? fma((T)2, du[0][0], d23) : (a == 1 ? s01 : s02);
      tau[1] = a == 1 ? fma((T)2, du[1][1], d23) : (a == 0 ? s01 : s12);
      tau[2] = a == 2 ? fma((T)2, du[2][2], d23) : (a == 0 ? s02 : s12);
      const T qa = fma(u, tau[0], fma(v, tau[1], fma(w, tau[2], dT[a])));
      f[1] = fma(iv, tau[0], f[1]);
      f[2] = fma(iv, tau[1], f[2]);
      f[3] = fma(iv, tau[2], f[3]);
      f[4] = fma(iv, qa, f[4]);
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) out[(long long)(a * 5 + c) * P + q] = f[c];
  }
}

// ------------------------------------------------------------------------------- k_rk

template <typename T, int ND>
__global__ void __launch_bounds__(512) k_rk(Geometry g, Physics ph, StepSched sc, const SubDev* __restrict__ subs,
                                            const T* __restrict__ Phi, const double* __restrict__ Uin0,
                                            double* __restrict__ Uout0, const double* __restrict__ ring, int in_ring,
                                            int out_ring, double* __restrict__ Q, double A, double B, double dt,
                                            int first, int last) {
  pdl_enter();
  sc = resolve(sc);
  const double* Uin = ring_or(Uin0, in_ring, ring, sc, 0);
  double* Uout = const_cast<double*>(ring_or(Uout0, out_ring, ring, sc, 1));
  const int sid = blockIdx.y;
  const SubDev d = subs[sid];
  if (!d.own) return;  // another process's sub-domain
  const int t = blockIdx.x * blockDim.x + threadIdx.x;  // own points of a sub-domain: < 2^31
  if (t >= d.sx * d.sy * d.sz) return;
  const int sxy = d.sx * d.sy, ck = t / sxy, r2 = t - ck * sxy, cj = r2 / d.sx, ci = r2 - cj * d.sx;
  const long long sty = d.ex, stz = (long long)d.ex * d.ey;
  const long long q = (long long)(ci + g.G) + sty * (cj + g.G) + stz * (ck + g.Gz);
  const long long gi = d.bbase + (long long)(d.ox + ci) + (long long)d.bnx * ((long long)(d.oy + cj) + (long long)d.bny * (d.oz + ck));
  const long long P = g.Ptot;
  const T* F = Phi + d.pbase;
  const long long st[3] = {1, sty, stz};
  const bool wallpt = d.wall && ((((d.wall >> 0) & 1) && ci == 0) || (((d.wall >> 1) & 1) && ci == d.sx - 1) ||
                                 (((d.wall >> 2) & 1) && cj == 0) || (((d.wall >> 3) & 1) && cj == d.sy - 1));
  // R = sum_a c1_a (Phi_{+1} - Phi_{-1}) + c2_a (Phi_{+2} - Phi_{-2}) as one FMA chain, times dt
  // (and J on a curvilinear block) once, for all five components before the first store (the
  // output may be a ring level the compiler cannot tell apart from Phi, so loads after a store
  // would wait for it)
  T k1[3], k2[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    k1[a] = (T)d.c1[a];
    k2[a] = (T)d.c2[a];
  }
  const double sdt = (d.mbase >= 0) ? dt * g.metric[d.mbase + 6 * d.mpl + (d.ox + ci + g.G) + (long long)d.mx * (d.oy + cj + g.G)] : dt;
  double dtR[5], qv[5], uv[5];
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    const T* Fx = F + (long long)c * P;
    T acc = k1[0] * (Fx[q + 1] - Fx[q - 1]);
    if (g.r == 2) acc = fma(k2[0], Fx[q + 2] - Fx[q - 2], acc);
#pragma unroll
    for (int a = 1; a < ND; ++a) {
      const T* Fa = F + (long long)(a * 5 + c) * P;
      acc = fma(k1[a], Fa[q + st[a]] - Fa[q - st[a]], acc);
      if (g.r == 2) acc = fma(k2[a], Fa[q + 2 * st[a]] - Fa[q - 2 * st[a]], acc);
    }
    dtR[c] = (double)acc * sdt;
  }
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    qv[c] = first ? 0.0 : Q[c * d.bN + gi];
    uv[c] = Uin[c * d.bN + gi];
  }
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    double qn = first ? dtR[c] : fma(A, qv[c], dtR[c]);
    double un = fma(B, qn, uv[c]);
    if (wallpt && c >= 1 && c <= 3) qn = un = 0.0;  // no-slip wall points keep zero momentum
    if (!last) Q[c * d.bN + gi] = qn;
    Uout[c * d.bN + gi] = un;
  }
}

// ------------------------------------------------------------------------------- compact scheme

// Sixth-order compact derivative (Eq. 2 with alpha = 1/3, a = 14/9, b = 1/9) of the combined
// fluxes Phi_axis along every owned line of a sub-domain, one thread per (line, component): the
// right side from the owned values and 2 halo values beyond each face, the closure values at the
// first halo point on each side by the explicit sixth-order central difference (45, -9, 1)/60h
// (which reads 4 halo values), then the tridiagonal solve (unit diagonal, off-diagonals alpha)
// with precomputed Thomas factors.  R = D_x Phi_x (axis 0), R += D_a Phi_a (axes 1, 2), FP64.
template <typename T, int axis>
__global__ void __launch_bounds__(128) k_compact_div(Geometry g, const SubDev* __restrict__ subs,
                                                     const T* __restrict__ Phi, double* __restrict__ R,
                                                     const double* __restrict__ cth, int Lmax) {
  const int sid = blockIdx.y;
  const SubDev d = subs[sid];
  if (!d.own) return;
  const int sz3[3] = {d.sx, d.sy, d.sz};
  constexpr int a1 = axis == 0 ? 1 : 0, a2 = axis == 2 ? 1 : 2;
  const int nl = sz3[a1] * sz3[a2];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 5 * nl) return;
  const int comp = t / nl, line = t - comp * nl;
  const int t1 = line % sz3[a1], t2 = line / sz3[a1];
  const int n = sz3[axis];
  const long long stp[3] = {1, d.ex, (long long)d.ex * d.ey};
  const long long st = stp[axis];
  int c0[3];
  c0[axis] = 0;
  c0[a1] = t1;
  c0[a2] = t2;
  const long long q0 = d.pbase + (long long)(c0[0] + g.G) + stp[1] * (c0[1] + g.G) + stp[2] * (c0[2] + g.Gz);
  const T* F = Phi + (long long)(axis * 5 + comp) * g.Ptot + q0;  // F[i * st]: point i of the line
  // own-point offsets in the state arrays (R)
  const long long r0 = d.bbase + (long long)comp * d.bN + (long long)(d.ox + c0[0]) +
                       (long long)d.bnx * ((long long)(d.oy + c0[1]) + (long long)d.bny * (d.oz + c0[2]));
  const long long gst[3] = {1, d.bnx, (long long)d.bnx * d.bny};
  const long long rs = gst[axis];
  const double h = 1.0 / (2.0 * d.c1[axis] * 3.0 / 4.0);  // c1 = (4/3 / 2) / h for the block's CD4 coefficients
  // the system is linear in its right side, so it is solved in units of cb = b / (4h): the right
  // side becomes (f_{i+2} - f_{i-2}) + 28 (f_{i+1} - f_{i-1}) (a / (2h) = 28 cb), the closures
  // (...) / (60 h) = 0.6 cb (...), and cb multiplies the solution once per point
  const double al = 1.0 / 3.0, cb = (1.0 / 9.0) / (4.0 * h);
  auto f = [&](int i) { return (double)F[(long long)i * st]; };
  const double dl = 0.6 * (45.0 * (f(0) - f(-2)) - 9.0 * (f(1) - f(-3)) + (f(2) - f(-4)));
  const double dr = 0.6 * (45.0 * (f(n + 1) - f(n - 1)) - 9.0 * (f(n + 2) - f(n - 2)) + (f(n + 3) - f(n - 3)));
  const double* cp = cth + (long long)n * 2 * Lmax;
  const double* im = cp + Lmax;
  // forward sweep: the eliminated right sides go to a per-thread array (local memory)
  double w[CFS_MAX_LINE];
  double prev = 0.0;
  for (int i = 0; i < n; ++i) {
    double rhs = fma(28.0, f(i + 1) - f(i - 1), f(i + 2) - f(i - 2));
    if (i == 0) rhs -= al * dl;
    if (i == n - 1) rhs -= al * dr;
    prev = (i == 0 ? rhs : rhs - al * prev) * __ldg(im + i);
    w[i] = prev;
  }
  // Phi_a = -F_a (k_flux stores the negated inviscid flux), so R = -sum_a D_a F_a = sum_a D_a Phi_a
  double x = prev;
  double* Rl = R + r0;
  if (axis == 0) Rl[(long long)(n - 1) * rs] = cb * x;
  else Rl[(long long)(n - 1) * rs] = fma(cb, x, Rl[(long long)(n - 1) * rs]);
  for (int i = n - 2; i >= 0; --i) {
    x = w[i] - __ldg(cp + i) * x;
    if (axis == 0) Rl[(long long)i * rs] = cb * x;
    else Rl[(long long)i * rs] = fma(cb, x, Rl[(long long)i * rs]);
  }
}

// Stage update from R: Q = A Q + dt R, U^(m) = U^(m-1) + B Q (Eq. 3, FP64).
__global__ void __launch_bounds__(512) k_rk_from_R(StepSched sc, const SubDev* __restrict__ subs,
                                                   const double* __restrict__ R, const double* __restrict__ Uin0,
                                                   double* __restrict__ Uout0, const double* __restrict__ ring,
                                                   int in_ring, int out_ring, double* __restrict__ Q, double A, double B,
                                                   double dt, int first, int last) {
  sc = resolve(sc);
  const double* Uin = ring_or(Uin0, in_ring, ring, sc, 0);
  double* Uout = const_cast<double*>(ring_or(Uout0, out_ring, ring, sc, 1));
  const int sid = blockIdx.y;
  const SubDev d = subs[sid];
  if (!d.own) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= d.sx * d.sy * d.sz) return;
  const int sxy = d.sx * d.sy, ck = t / sxy, r2 = t - ck * sxy, cj = r2 / d.sx, ci = r2 - cj * d.sx;
  const long long gi = d.bbase + (long long)(d.ox + ci) + (long long)d.bnx * ((long long)(d.oy + cj) + (long long)d.bny * (d.oz + ck));
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    const double dtR = dt * R[c * d.bN + gi];
    const double qn = first ? dtR : fma(A, Q[c * d.bN + gi], dtR);
    if (!last) Q[c * d.bN + gi] = qn;
    Uout[c * d.bN + gi] = fma(B, qn, Uin[c * d.bN + gi]);
  }
}

static inline unsigned nblk(long long n, int b) { return (unsigned)((n + b - 1) / b); }

#define TIMED(tm, kind, launch)              \
  do {                                       \
    if (tm) tm->rec(tm->self, kind, 1);      \
    launch;                                  \
    if (tm) tm->rec(tm->self, kind, 0);      \
  } while (0)

template <typename T>
static int stage_impl(const Geometry& g, const Physics& ph, const StepSched& sc, const StageLaunch& a,
                      cudaStream_t st, long long* launches, const Timer* tm) {
  const int B = (a.threads == 128 || a.threads == 512) ? a.threads : 256;
  dim3 gf(nblk(a.max_flux, B), g.nsub), gr(nblk(a.max_own, B), g.nsub);
  {
    const unsigned own_blocks = nblk(a.max_own, B);
    const unsigned nb = own_blocks * (unsigned)g.nsub + nblk(a.nhalo, B);
    TIMED(tm, 0, (launch_pdl(k_view<T>, dim3(nb), dim3(B), 0, st, g, ph, sc, a.Uin, a.ring, a.in_ring, a.subs,
                             (const int2*)a.halo, a.nhalo, (T*)a.Wp, a.stage, a.s, (int)own_blocks)));
  }
  if (a.compact) {
    // compact scheme: fluxes, then one line-solve launch per axis into R, then the update
    const long long nl = 5LL * a.Lmax * a.Lmax;
    const dim3 gl(nblk(nl, 128), g.nsub);
    if (g.ndim == 3) {
      TIMED(tm, 1, ((g.metric ? k_flux<T, 3, true> : k_flux<T, 3, false>)<<<gf, B, 0, st>>>(g, ph, a.subs, (const T*)a.Wp, (T*)a.Phi)));
      TIMED(tm, 2, (k_compact_div<T, 0><<<gl, 128, 0, st>>>(g, a.subs, (const T*)a.Phi, a.R, a.cthomas, a.Lmax)));
      TIMED(tm, 2, (k_compact_div<T, 1><<<gl, 128, 0, st>>>(g, a.subs, (const T*)a.Phi, a.R, a.cthomas, a.Lmax)));
      TIMED(tm, 2, (k_compact_div<T, 2><<<gl, 128, 0, st>>>(g, a.subs, (const T*)a.Phi, a.R, a.cthomas, a.Lmax)));
    } else {
      TIMED(tm, 1, ((g.metric ? k_flux<T, 2, true> : k_flux<T, 2, false>)<<<gf, B, 0, st>>>(g, ph, a.subs, (const T*)a.Wp, (T*)a.Phi)));
      TIMED(tm, 2, (k_compact_div<T, 0><<<gl, 128, 0, st>>>(g, a.subs, (const T*)a.Phi, a.R, a.cthomas, a.Lmax)));
      TIMED(tm, 2, (k_compact_div<T, 1><<<gl, 128, 0, st>>>(g, a.subs, (const T*)a.Phi, a.R, a.cthomas, a.Lmax)));
    }
    TIMED(tm, 2, (k_rk_from_R<<<gr, B, 0, st>>>(sc, a.subs, a.R, a.Uin, a.Uout, a.ring, a.in_ring, a.out_ring, a.Q, a.A,
                                                a.B, a.dt, a.first, a.last)));
    if (launches) *launches += 1 + 1 + g.ndim + 1;
    return (int)cudaGetLastError();
  }
  if (g.ndim == 3) {
    TIMED(tm, 1, (launch_pdl(g.metric ? k_flux<T, 3, true> : k_flux<T, 3, false>, gf, dim3(B), 0, st, g, ph, a.subs, (const T*)a.Wp, (T*)a.Phi)));
    TIMED(tm, 2, (launch_pdl(k_rk<T, 3>, gr, dim3(B), 0, st, g, ph, sc, a.subs, (const T*)a.Phi, a.Uin, a.Uout, a.ring,
                             a.in_ring, a.out_ring, a.Q, a.A, a.B, a.dt, a.first, a.last)));
  } else {
    TIMED(tm, 1, (launch_pdl(g.metric ? k_flux<T, 2, true> : k_flux<T, 2, false>, gf, dim3(B), 0, st, g, ph, a.subs, (const T*)a.Wp, (T*)a.Phi)));
    TIMED(tm, 2, (launch_pdl(k_rk<T, 2>, gr, dim3(B), 0, st, g, ph, sc, a.subs, (const T*)a.Phi, a.Uin, a.Uout, a.ring,
                             a.in_ring, a.out_ring, a.Q, a.A, a.B, a.dt, a.first, a.last)));
  }
  if (launches) *launches += 3;
  return (int)cudaGetLastError();
}

int launch_stage(const Geometry& g, const Physics& ph, const StepSched& sc, const StageLaunch& a, int precision,
                 void* stream, long long* launches, const Timer* tm) {
  cudaStream_t st = (cudaStream_t)stream;
  if (precision == 1) return stage_impl<float>(g, ph, sc, a, st, launches, tm);
  return stage_impl<double>(g, ph, sc, a, st, launches, tm);
}

// ------------------------------------------------------------------------------- k_filter

// One CTA per (variable, line segment of one sub-domain, group of LN lines); one thread per line
// in the solve.  Lines along `axis`; the two other axes are f1 (x unless axis is x) and f2.  The
// CTA first stages the 11-point windows of all its lines -- own values, and halo values by the
// schedule (SA: live neighbour; AT: extrapolation to t_{n+1} with the weights c(k+1) in FP64;
// AS: the latest delayed level) -- in shared memory with coalesced loads (consecutive threads
// along the line for the x pass, across lines for y and z), solves each line from there, and
// stores the result with the same pattern.  Right side: sum_n (a_n/2)(f_{i+n} + f_{i-n});
// Dirichlet closure f^_{-1} = f_{-1}, f^_L = f_L; Thomas factors precomputed per line length.
struct FilterTile {
  int LN;  // lines per CTA
  int TW;  // row stride in doubles (odd: 64-bit accesses of a warp's rows hit distinct banks)
};

__host__ __device__ inline FilterTile filter_tile(int Lmax) {
  FilterTile t;
  t.TW = (Lmax + 10) | 1;
  t.LN = 128;
  while (t.LN > 32 && (size_t)(t.LN + 1) * t.TW * 12 > 200 * 1024) t.LN /= 2;
  return t;
}

// Shared memory of k_filter: the line tiles ([LN][TW] doubles, or floats in the FP32 form) and the
// TW position offsets.
__host__ __device__ inline size_t filter_tile_doubles(const FilterTile& t, int precision) {
  return precision == 1 ? ((size_t)t.LN * t.TW + 1) / 2 : (size_t)t.LN * t.TW;
}
__host__ __device__ inline size_t filter_smem_bytes(int Lmax, int precision) {
  const FilterTile t = filter_tile(Lmax);
  return (filter_tile_doubles(t, precision) + t.TW) * 8;
}

template <typename T, int axis>
__global__ void __launch_bounds__(128) k_filter(Geometry g, StepSched sc, FilterLaunch f) {
  pdl_enter();
  sc = resolve(sc);
  if (f.only_sync && sc.mode != 0) return;
  constexpr bool F32 = std::is_same<T, float>::value;
  const double* __restrict__ Uin = ring_or(f.Uin, f.in_ring, f.ring, sc, 0);
  double* __restrict__ Uout = const_cast<double*>(ring_or(f.Uout, f.out_ring, f.ring, sc, 1));
  constexpr int f1 = (axis == 0) ? 1 : 0;
  constexpr int f2 = (axis == 2) ? 1 : 2;
  const int n[3] = {f.nx, f.ny, f.nz};
  const long long strides[3] = {1, f.nx, (long long)f.nx * f.ny};
  const FilterTile tl = filter_tile(f.Lt);
  const int LN = tl.LN, TW = tl.TW;
  extern __shared__ __align__(16) double fsm[];
  // [LN][TW] window slots (positions -5 .. len+4): FP64 values, or in the FP32 form FP32 offsets
  // from the line's first own value (staged converted, so a line needs 4 bytes per slot)
  double* tile = fsm;
  float* ftile = reinterpret_cast<float*>(fsm);
  long long* sPos = reinterpret_cast<long long*>(fsm + filter_tile_doubles(tl, F32 ? 1 : 0));  // [TW] offsets

  const long long nl = (long long)n[f1] * n[f2];
  const int groups = (int)((nl + LN - 1) / LN);
  int b = blockIdx.x;
  const int grp = b % groups;
  b /= groups;
  const int seg = b % f.P[axis];
  const int var = b / f.P[axis];
  const int off = f.axis_off[axis][seg], len = f.axis_len[axis][seg];
  const int W = len + 10;
  const long long l0 = (long long)grp * LN;
  const int nlines = (int)min((long long)LN, nl - l0);
  const long long st = strides[axis];
  const long long lvN = 5 * g.N;
  // per-CTA tables: line bases and face delays, offsets of the window positions along the line,
  // and ring-level offsets per (delay, level)
  __shared__ long long sBase[128];
  __shared__ long long sLev[(CFS_MAX_DELAY + 2) * CFS_MAX_LEVELS];
  __shared__ int sKd[2][128];
  __shared__ int sSid[128], sT1[128], sT2[128];  // blocks with a gather map: the line's sub-domain and position
  __shared__ double sRef[128];                   // FP32 form: the line's first own value
  __shared__ unsigned char sOk[128];             // the line belongs to a sub-domain computed here
  const bool gmap = f.ebase >= 0;
  for (int t = threadIdx.x; t < nlines; t += blockDim.x) {
    const long long t12 = l0 + t;
    const int t1 = (int)(t12 % n[f1]), t2 = (int)(t12 / n[f1]);
    sBase[t] = f.bbase + (long long)var * f.bN + (long long)t1 * strides[f1] + (long long)t2 * strides[f2];
    sOk[t] = 1;
    if (f.subs) {  // partitioned context: skip the lines of another process's sub-domains
      int sidx[3];
      sidx[axis] = seg;
      sidx[f1] = f.owner[f1][t1];
      sidx[f2] = f.owner[f2][t2];
      sOk[t] = (unsigned char)f.subs[f.sid0 + sidx[0] + f.P[0] * (sidx[1] + f.P[1] * sidx[2])].own;
    }
    int kl = 0, kr = 0;
    if (sc.mode != 0 || gmap) {
      int sidx[3];
      sidx[axis] = seg;
      sidx[f1] = f.owner[f1][t1];
      sidx[f2] = f.owner[f2][t2];
      const int sid = f.sid0 + sidx[0] + f.P[0] * (sidx[1] + f.P[1] * sidx[2]);
      // a sub-domain face on a physical block boundary has no neighbouring PE and no delay
      const bool pl = seg == 0 && ((f.phys >> (2 * axis)) & 1);
      const bool pr = seg == f.P[axis] - 1 && ((f.phys >> (2 * axis + 1)) & 1);
      if (sc.mode != 0) {
        kl = pl ? 0 : face_delay(sc, sid, 2 * axis);
        kr = pr ? 0 : face_delay(sc, sid, 2 * axis + 1);
      }
      sSid[t] = sid;
      sT1[t] = t1;
      sT2[t] = t2;
    }
    sKd[0][t] = kl;
    sKd[1][t] = kr;
    if (F32 && sOk[t]) sRef[t] = Uin[sBase[t] + (long long)off * st];
  }
  for (int t = threadIdx.x; t < W; t += blockDim.x) sPos[t] = (long long)wrapc(off + t - 5, n[axis]) * st;
  if (sc.mode != 0) {
    const int nk = (int)min((long long)CFS_MAX_DELAY + 1, max(sc.cap, 0LL) + 1);
    for (int t = threadIdx.x; t < nk * sc.C; t += blockDim.x) {
      const int kd = t / sc.C, l = t % sc.C;
      sLev[t] = (long long)((sc.n - kd - l) % sc.R) * lvN;
    }
  }
  __syncthreads();

  // ---- stage the windows: value at window slot i (position i - 5) of line `line`
  // beyond a non-periodic block face: the face's sources -- own ones current, a neighbouring PE's
  // by the mode, far-field constants
  auto gather_value = [&](int line, int pos, int u) -> double {
    int cc[3];
    cc[axis] = u;
    cc[f1] = sT1[line];
    cc[f2] = sT2[line];
    const int ei = g.emap[f.ebase + (cc[0] + g.GE) + (long long)f.gmx * ((cc[1] + g.GE) + (long long)f.gmy * cc[2])];
    const GatherEntry& E = g.gent[ei];
    const int kd = sKd[pos < 0 ? 0 : 1][line];
    double v = E.cst[var];
    for (int t = 0; t < E.nt; ++t) {
      const bool own = !(E.flags[t] & 2) && E.sid[t] == sSid[line];
      const double sg = ((E.flags[t] & 1) && var >= 1 && var <= 3) ? -E.w[t] : E.w[t];
      const long long o = E.off[t] + (long long)var * E.bN[t];
      double x;
      if (own || sc.mode == 0) {
        x = Uin[o];
      } else if (sc.mode == 2) {
        x = f.ring[sLev[kd * sc.C] + o];
      } else {
        x = 0.0;
        for (int l = 0; l < sc.C; ++l) x = fma(__ldg(sc.Wf + kd * sc.C + l), f.ring[sLev[kd * sc.C + l] + o], x);
      }
      v = fma(sg, x, v);
    }
    return v;
  };
  // halo slot inside the block: SA the neighbour's value, AS the latest visible level, AT the
  // extrapolation to t_{n+1} with the weights c(k+1), in FP64
  auto halo_value = [&](int line, int pos, long long gi) -> double {
    const int kd = sKd[pos < 0 ? 0 : 1][line];
    if (sc.mode == 2) return f.ring[sLev[kd * sc.C] + gi];
    double v = 0.0;
    for (int l = 0; l < sc.C; ++l) v = fma(__ldg(sc.Wf + kd * sc.C + l), f.ring[sLev[kd * sc.C + l] + gi], v);
    return v;
  };
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  if (!F32) {
    // FP64 values; plain copies of U or of one ring level through cp.async
    auto stage = [&](int line, int i) {
      const int pos = i - 5;
      const long long gi = sBase[line] + sPos[i];
      double* dst = tile + line * TW + i;
      const int u = off + pos;
      if (gmap && axis < 2 && (u < 0 || u >= n[axis])) *dst = gather_value(line, pos, u);
      else if ((pos >= 0 && pos < len) || sc.mode == 0) cp_async8(dst, Uin + gi);
      else if (sc.mode == 2) cp_async8(dst, f.ring + sLev[sKd[pos < 0 ? 0 : 1][line] * sc.C] + gi);
      else *dst = halo_value(line, pos, gi);
    };
    if (axis == 0) {
      // own points: a warp per line, lanes along it (contiguous in memory); the 10 window points
      // outside the segment: a thread per line, so that no warp mixes copies with extrapolations
      for (int line = warp; line < nlines; line += nwarp)
        if (sOk[line])
          for (int i = 5 + lane; i < 5 + len; i += 32) cp_async8(tile + line * TW + i, Uin + sBase[line] + sPos[i]);
      for (int line = threadIdx.x; line < nlines; line += blockDim.x)
        if (sOk[line])
          for (int h = 0; h < 10; ++h) stage(line, h < 5 ? h : len + h);
    } else {  // threads across lines (consecutive x)
      for (int line = threadIdx.x; line < nlines; line += blockDim.x)
        if (sOk[line])
          for (int i = 0; i < W; ++i) stage(line, i);
    }
  } else {
    // FP32 form: every value converted on arrival to its offset from the line's first own value
    // (dev_fast: the FP64 difference rounded once), so a slot is 4 bytes
    auto value = [&](int line, int i) -> double {
      const int pos = i - 5;
      const long long gi = sBase[line] + sPos[i];
      const int u = off + pos;
      if (gmap && axis < 2 && (u < 0 || u >= n[axis])) return gather_value(line, pos, u);
      if ((pos >= 0 && pos < len) || sc.mode == 0) return Uin[gi];
      return halo_value(line, pos, gi);
    };
    auto put = [&](int line, int i, double v) {
      const double ref = sRef[line];
      const float rh = d2f_fast(ref), rl = dev_fast(ref, rh, 0.f);
      ftile[line * TW + i] = dev_fast(v, rh, rl);
    };
    if (axis == 0) {
      for (int line = warp; line < nlines; line += nwarp)
        if (sOk[line])
          for (int i = 5 + lane; i < 5 + len; i += 32) put(line, i, Uin[sBase[line] + sPos[i]]);
      for (int line = threadIdx.x; line < nlines; line += blockDim.x)
        if (sOk[line])
          for (int h = 0; h < 10; ++h) {
            const int i = h < 5 ? h : len + h;
            put(line, i, value(line, i));
          }
    } else {
      for (int line = threadIdx.x; line < nlines; line += blockDim.x)
        if (sOk[line])
          for (int i = 0; i < W; ++i) put(line, i, value(line, i));
    }
  }
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();

  // ---- one line per thread
  const int line = threadIdx.x;
  if (line < nlines && sOk[line]) {
    double* row = tile + line * TW;
    const double* cp = f.thomas + (long long)len * 2 * f.Lmax;
    const double* im = cp + f.Lmax;
    if (!F32) {
      // FP64: the system as written, alpha f^_{i-1} + f^_i + alpha f^_{i+1} = rhs_i; the forward
      // sweep parks d_i in slot i (position i - 5, no longer read), back substitution overwrites
      const double al = f.alpha;
      double win[11];
#pragma unroll
      for (int m = 0; m < 11; ++m) win[m] = row[m];
      const double hm1 = row[4], hpl = row[len + 5];
      double dprev = 0.0;
      #pragma unroll 4
      for (int i = 0; i < len; ++i) {
        double rhs = f.h[0] * win[5];
#pragma unroll
        for (int m = 1; m <= 5; ++m) rhs = fma(f.h[m], win[5 + m] + win[5 - m], rhs);
        if (i == 0) rhs -= al * hm1;
        if (i == len - 1) rhs -= al * hpl;
        const double dcur = (i == 0 ? rhs : rhs - al * dprev) * __ldg(im + i);
        row[i] = dcur;
        dprev = dcur;
#pragma unroll
        for (int m = 0; m < 10; ++m) win[m] = win[m + 1];
        if (i + 11 < W) win[10] = row[i + 11];
      }
      double xnext = dprev;
      #pragma unroll 4
      for (int i = len - 2; i >= 0; --i) {
        const double x = row[i] - __ldg(cp + i) * xnext;
        row[i] = x;
        xnext = x;
      }
    } else {
      // FP32 form: solve for the increment d = f^ - f.  Its right side is
      // (a_1/2 - alpha) D_1 + sum_{n>=2} (a_n/2) D_n with D_n = f_{i+n} + f_{i-n} - 2 f_i (exact
      // algebra, using sum a_n = 1 + 2 alpha), the Dirichlet closure becomes d = 0 at the first
      // halo point, and the values enter as the FP32 offsets staged from an FP64 reference of the
      // line, so FP32 rounding never acts on the full magnitude of the state.  The forward sweep
      // parks its d_i in slot i (no longer read), back substitution leaves the increment of point
      // i there; the store adds it to the FP64 value.
      float* frow = ftile + line * TW;
      const float* cp32 = f.thomas32 + (long long)len * 2 * f.Lmax;  // the factors in FP32
      const float* im32 = cp32 + f.Lmax;
      float win[11];
#pragma unroll
      for (int m = 0; m < 11; ++m) win[m] = frow[m];
      const float b1 = (float)f.b1, al32 = (float)f.alpha;
      float hm[6];
#pragma unroll
      for (int m = 2; m <= 5; ++m) hm[m] = (float)f.h[m];
      float dprev = 0.f;
      #pragma unroll 4
      for (int i = 0; i < len; ++i) {
        const float c2 = 2.f * win[5];
        float rhs = b1 * (win[6] + win[4] - c2);
#pragma unroll
        for (int m = 2; m <= 5; ++m) rhs = fmaf(hm[m], win[5 + m] + win[5 - m] - c2, rhs);
        const float dcur = (i == 0 ? rhs : rhs - al32 * dprev) * __ldg(im32 + i);
        frow[i] = dcur;
        dprev = dcur;
#pragma unroll
        for (int m = 0; m < 10; ++m) win[m] = win[m + 1];
        if (i + 11 < W) win[10] = frow[i + 11];
      }
      float xnext = dprev;
      #pragma unroll 4
      for (int i = len - 2; i >= 0; --i) {
        const float x = frow[i] - __ldg(cp32 + i) * xnext;
        frow[i] = x;
        xnext = x;
      }
    }
  }
  __syncthreads();

  // ---- store the own points; no-slip wall points keep zero momentum
  const bool wz = f.wall && var >= 1 && var <= 3;
  auto wall_pt = [&](int ln, int i) {
    const int u = off + i, a1 = sT1[ln], a2 = sT2[ln];
    return (((f.wall >> (2 * axis)) & 1) && u == 0) || (((f.wall >> (2 * axis + 1)) & 1) && u == n[axis] - 1) ||
           (((f.wall >> (2 * f1)) & 1) && a1 == 0) || (((f.wall >> (2 * f1 + 1)) & 1) && a1 == n[f1] - 1) ||
           (((f.wall >> (2 * f2)) & 1) && a2 == 0) || (((f.wall >> (2 * f2 + 1)) & 1) && a2 == n[f2] - 1);
  };
  // the filtered value of point i: slot i (FP64), or the FP64 value plus the FP32 increment
  auto result = [&](int ln, int i, long long gi) -> double {
    if (wz && wall_pt(ln, i)) return 0.0;
    if (F32) return Uin[gi] + f2d_fast(ftile[ln * TW + i]);
    return tile[ln * TW + i];
  };
  if (axis == 0) {
    for (int ln = warp; ln < nlines; ln += nwarp)
      if (sOk[ln])
        for (int i = lane; i < len; i += 32) {
          const long long gi = sBase[ln] + sPos[i + 5];
          Uout[gi] = result(ln, i, gi);
        }
  } else {
    for (int ln = threadIdx.x; ln < nlines; ln += blockDim.x)
      if (sOk[ln])
        for (int i = 0; i < len; ++i) {
          const long long gi = sBase[ln] + sPos[i + 5];
          Uout[gi] = result(ln, i, gi);
        }
  }
}

__global__ void k_round_table(const double* __restrict__ x, float* __restrict__ y, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = d2f_fast(x[i]);
}

int launch_round_table(const double* x, float* y, long long n, void* stream) {
  if (n > 0) k_round_table<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(x, y, n);
  return (int)cudaGetLastError();
}

// The shared-memory opt-in of the line-filter kernels is a per-device attribute shared by every
// context of the process: it only ever rises (to the largest size a context on the device has
// needed), so a context with shorter lines cannot lower it under another one still stepping.
int filter_prepare(int Lmax, int precision) {
  const size_t sm = filter_smem_bytes(Lmax, precision);
  if (sm > 227 * 1024) return (int)cudaErrorInvalidValue;
  static std::mutex mu;
  static int set_to[64][2] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return (int)e;
  if (dev < 0 || dev >= 64) return (int)cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(mu);
  int& cur = set_to[dev][precision == 1 ? 1 : 0];
  if ((int)sm <= cur) return 0;
  const int b = (int)sm;
  if (precision == 1) {
    e = cudaFuncSetAttribute(k_filter<float, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_filter<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_filter<float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  } else {
    e = cudaFuncSetAttribute(k_filter<double, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_filter<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_filter<double, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  }
  if (e == cudaSuccess) cur = b;
  return (int)e;
}

int launch_filter(const Geometry& g, const StepSched& sc, const FilterLaunch& f, int axis, int precision,
                  void* stream, long long* launches, const Timer* tm) {
  const int n[3] = {f.nx, f.ny, f.nz};
  const int f1 = (axis == 0) ? 1 : 0;
  const int f2 = (axis == 2) ? 1 : 2;
  const FilterTile tl = filter_tile(f.Lt);
  const long long nl = (long long)n[f1] * n[f2];
  const unsigned nb = (unsigned)(5LL * f.P[axis] * ((nl + tl.LN - 1) / tl.LN));
  const size_t sm = filter_smem_bytes(f.Lt, precision);
  cudaStream_t st = (cudaStream_t)stream;
  if (tm) tm->rec(tm->self, 3, 1);
  if (precision == 1) {
    if (axis == 0) k_filter<float, 0><<<nb, 128, sm, st>>>(g, sc, f);
    else if (axis == 1) k_filter<float, 1><<<nb, 128, sm, st>>>(g, sc, f);
    else k_filter<float, 2><<<nb, 128, sm, st>>>(g, sc, f);
  } else {
    if (axis == 0) launch_pdl(k_filter<double, 0>, dim3(nb), dim3(128), sm, st, g, sc, f);
    else if (axis == 1) launch_pdl(k_filter<double, 1>, dim3(nb), dim3(128), sm, st, g, sc, f);
    else launch_pdl(k_filter<double, 2>, dim3(nb), dim3(128), sm, st, g, sc, f);
  }
  if (tm) tm->rec(tm->self, 3, 0);
  if (launches) *launches += 1;
  return (int)cudaGetLastError();
}

// ------------------------------------------------------------------------------- diagnostics

// Velocity component c at (x, y, z) of a block with periodic wrap.
__device__ __forceinline__ double vel_at(const double* U, const DiagBlock& b, int x, int y, int z, int c) {
  const long long gi = b.bbase + (long long)wrapc(x, b.nx) + (long long)b.nx * ((long long)wrapc(y, b.ny) + (long long)b.ny * wrapc(z, b.nz));
  return U[(1 + c) * b.bN + gi] / U[gi];
}

__global__ void __launch_bounds__(256) k_diag(DiagBlock b, const double* __restrict__ U, double* __restrict__ partial) {
  double acc[DIAG_NQ] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  const int ndim = b.nz > 1 ? 3 : 2;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < b.bN; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % b.nx), y = (int)((i / b.nx) % b.ny), z = (int)(i / ((long long)b.nx * b.ny));
    if (b.subs && !b.subs[b.sid0 + b.owner[0][x] + b.P[0] * (b.owner[1][y] + b.P[1] * b.owner[2][z])].own) continue;
    const long long mq = (long long)(x + b.G) + (long long)b.mx * (y + b.G);  // metric plane index
    const double dV = b.M ? b.M[5 * b.mpl + mq] : b.dV;  // cell volume (J^-1 on a curvilinear grid)
    double u[5];
    for (int v = 0; v < 5; ++v) {
      u[v] = U[b.bbase + v * b.bN + i];
      if (!isfinite(u[v])) acc[7] = 1.0;
      acc[2 + v] += u[v] * dV;
    }
    const double rho = u[0];
    const double vx = u[1] / rho, vy = u[2] / rho, vz = u[3] / rho;
    acc[0] += 0.5 * rho * (vx * vx + vy * vy + vz * vz) * dV;
    // enstrophy only where the CD stencils stay in the block or cross periodic faces
    if (b.nonper) {
      const int c3[3] = {x, y, z}, n3[3] = {b.nx, b.ny, b.nz};
      bool inner = true;
      for (int a = 0; a < ndim; ++a) {
        if (((b.nonper >> (2 * a)) & 1) && c3[a] < b.rs) inner = false;
        if (((b.nonper >> (2 * a + 1)) & 1) && c3[a] > n3[a] - 1 - b.rs) inner = false;
      }
      if (!inner) continue;
    }
    acc[8] += dV;
    // vorticity by the CD scheme
    double dv[3][3];
    for (int c = 0; c < 3; ++c)
      for (int a = 0; a < 3; ++a) {
        if (a >= ndim) { dv[c][a] = 0.0; continue; }
        const int ex = a == 0, ey = a == 1, ez = a == 2;
        double dd = b.c1[a] * (vel_at(U, b, x + ex, y + ey, z + ez, c) - vel_at(U, b, x - ex, y - ey, z - ez, c));
        if (b.c2[a] != 0.0)
          dd += b.c2[a] * (vel_at(U, b, x + 2 * ex, y + 2 * ey, z + 2 * ez, c) -
                           vel_at(U, b, x - 2 * ex, y - 2 * ey, z - 2 * ez, c));
        dv[c][a] = dd;
      }
    if (b.M) {  // index-space derivatives -> physical: d/dx_j = J sum_k (metric row k)_j d/dxi_k
      const double J = b.M[6 * b.mpl + mq];
      const double m[3][3] = {{b.M[mq], b.M[b.mpl + mq], 0.0}, {b.M[2 * b.mpl + mq], b.M[3 * b.mpl + mq], 0.0},
                              {0.0, 0.0, b.M[4 * b.mpl + mq]}};
      double dp[3][3];
      for (int c = 0; c < 3; ++c)
        for (int j = 0; j < 3; ++j) dp[c][j] = J * (m[0][j] * dv[c][0] + m[1][j] * dv[c][1] + m[2][j] * dv[c][2]);
      for (int c = 0; c < 3; ++c)
        for (int j = 0; j < 3; ++j) dv[c][j] = dp[c][j];
    }
    const double wx = dv[2][1] - dv[1][2], wy = dv[0][2] - dv[2][0], wz = dv[1][0] - dv[0][1];
    acc[1] += 0.5 * rho * (wx * wx + wy * wy + wz * wz) * dV;
  }
  // block reduction: warp shuffles, then one warp over the warp sums
  __shared__ double sh[DIAG_NQ][8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int c = 0; c < DIAG_NQ; ++c) {
    double v = acc[c];
    for (int o = 16; o > 0; o >>= 1) {
      const double other = __shfl_down_sync(0xffffffffu, v, o);
      v = (c == 7) ? fmax(v, other) : v + other;
    }
    if (lane == 0) sh[c][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < DIAG_NQ) {
    const int c = threadIdx.x;
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v = (c == 7) ? fmax(v, sh[c][w]) : v + sh[c][w];
    partial[(long long)blockIdx.x * DIAG_NQ + c] = v;
  }
}

// Deterministic second pass: one thread per quantity sums the block partials in block order.
// K is a volume average (sum of value x cell volume over the total volume), the enstrophy an
// average over the volume of the points it covers.
__global__ void k_diag_final(const double* __restrict__ partial, int nblocks, double* __restrict__ out, double volume) {
  const int c = threadIdx.x;
  if (c >= 8) return;
  double v = 0.0, ve = 0.0;
  for (int b = 0; b < nblocks; ++b) {
    v = (c == 7) ? fmax(v, partial[(long long)b * DIAG_NQ + c]) : v + partial[(long long)b * DIAG_NQ + c];
    ve += partial[(long long)b * DIAG_NQ + 8];
  }
  if (c == 0) v /= volume;
  if (c == 1) v = ve > 0.0 ? v / ve : 0.0;
  out[c] = v;
}

int launch_diagnostics_block(const Geometry& g, const DiagBlock& b, const double* U, double* partial, int row0,
                             int nblocks, void* stream) {
  k_diag<<<nblocks, 256, 0, (cudaStream_t)stream>>>(b, U, partial + (long long)row0 * DIAG_NQ);
  return (int)cudaGetLastError();
}

__global__ void k_advance_step(long long* dn) {
  pdl_enter();
  if (threadIdx.x == 0 && blockIdx.x == 0) *dn += 1;
}

__global__ void k_eval_power(const double* __restrict__ x, double a, double* __restrict__ y, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = pow_tab(x[i], a);
}

// The tables of pow_tab in the current device's copy of the __device__ array, once per device
// (each device that runs the power holds its own copy).  A failed upload is not remembered: the
// next call on that device tries again.
int pow_tables_init() {
  constexpr int kMaxDev = 64;
  static std::mutex mu;
  static bool done[kMaxDev] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return (int)e;
  if (dev < 0 || dev >= kMaxDev) return (int)cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev]) return 0;
  double t[3 * 64];
  for (int j = 0; j < 64; ++j) {
    t[j] = 128.0 / (129.0 + 2.0 * j);  // 1/c_j, c_j = (129 + 2j)/128
    t[64 + j] = (double)log1pl((long double)(2 * j + 1) / 128.0L);
    t[128 + j] = (double)exp2l((long double)j / 64.0L);
  }
  e = cudaMemcpyToSymbol(g_pow_tab, t, sizeof(t));
  if (e != cudaSuccess) return (int)e;
  done[dev] = true;
  return 0;
}

int launch_eval_power(const double* x, double a, double* y, long long n, void* stream) {
  if (int rc = pow_tables_init()) return rc;
  if (n > 0) k_eval_power<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(x, a, y, n);
  return (int)cudaGetLastError();
}

// FP64 pipe probe: every thread runs 8 independent DFMA chains of `iters` steps (x <- x a + b,
// with a = 1 - 2^-40 and b chosen so the values stay bounded) and writes one sum, so the pipe
// has independent work and nothing is folded away.  DFMAs executed = blocks x threads x iters x 8.
__global__ void __launch_bounds__(256) k_fp64_probe(double* __restrict__ sink, int iters, double a, double b) {
  double x[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) x[c] = 1.0 + (threadIdx.x + c) * 1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = fma(x[c], a, b);
  }
  double t = 0.0;
#pragma unroll
  for (int c = 0; c < 8; ++c) t += x[c];
  sink[(long long)blockIdx.x * blockDim.x + threadIdx.x] = t;
}

// Self-test of the bounded waits the tensor-core kernels use: an mbarrier expecting one arrival
// that never comes; every thread polls it at most limit + 1 times, gives up, and thread 0 records
// the give-up in the status word the host reads (CFS_ETIMEOUT).  Nothing is left in flight.
__global__ void k_wait_check(int* status, unsigned limit) {
  __shared__ unsigned long long bar;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"((unsigned)__cvta_generic_to_shared(&bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  const bool ok = mbar_wait_bounded(&bar, 0u, limit);
  if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicOr(status, 1);
}

int launch_wait_check(int* status, unsigned limit, void* stream) {
  k_wait_check<<<1, 128, 0, (cudaStream_t)stream>>>(status, limit);
  return (int)cudaGetLastError();
}

int launch_fp64_probe(double* sink, int blocks, int iters, void* stream) {
  k_fp64_probe<<<blocks, 256, 0, (cudaStream_t)stream>>>(sink, iters, 1.0 - 0x1p-40, 0x1p-41);
  return (int)cudaGetLastError();
}

// ------------------------------------------------------------------------------- strip exchange

// Boundary strips of a partitioned context: one thread per (entry, variable), entries of a plan
// in order, 5 values per entry (the layout sent to a peer).
__global__ void k_strip_pack(const double* __restrict__ U, const long long* __restrict__ off, const int* __restrict__ bN,
                             long long n, double* __restrict__ buf) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 5 * n) return;
  const long long i = t / 5;
  const int v = (int)(t - 5 * i);
  buf[t] = U[off[i] + (long long)v * bN[i]];
}

__global__ void k_strip_unpack(double* __restrict__ U, const long long* __restrict__ off, const int* __restrict__ bN,
                               long long n, const double* __restrict__ buf) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 5 * n) return;
  const long long i = t / 5;
  const int v = (int)(t - 5 * i);
  U[off[i] + (long long)v * bN[i]] = buf[t];
}

int launch_strip_pack(const double* U, const long long* off, const int* bN, long long n, double* buf, void* stream) {
  if (n > 0) k_strip_pack<<<(unsigned)((5 * n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(U, off, bN, n, buf);
  return (int)cudaGetLastError();
}

int launch_strip_unpack(double* U, const long long* off, const int* bN, long long n, const double* buf, void* stream) {
  if (n > 0) k_strip_unpack<<<(unsigned)((5 * n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(U, off, bN, n, buf);
  return (int)cudaGetLastError();
}

int launch_advance_step(long long* dn, void* stream) {
  launch_pdl(k_advance_step, dim3(1), dim3(32), 0, (cudaStream_t)stream, dn);
  return (int)cudaGetLastError();
}

int launch_diagnostics_final(const double* partial, int nrows, double* out, double volume, void* stream) {
  k_diag_final<<<1, 32, 0, (cudaStream_t)stream>>>(partial, nrows, out, volume);
  return (int)cudaGetLastError();
}

}  // namespace cfs
