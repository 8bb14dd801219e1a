// topology.cpp -- host side of connected multi-block grids: validation of the block faces, the
// gather entries of the points beyond non-periodic block faces, and the metric planes of
// curvilinear blocks continued across their faces.
//
// Conventions (the readings of the paper's multi-block grid, whose topology and boundary
// closures it does not print): blocks are node-disjoint -- the first point beyond a block face
// is the neighbour's first point inside its face; an interface joins in-plane faces (x or y) with
// the tangential in-plane index running the same way or reversed; spanwise counts may differ, a
// receiving point then takes the neighbour's values at its own spanwise position by four-point
// Lagrange interpolation (exact positions: the point itself).  A no-slip adiabatic wall mirrors
// the state about the face with the momentum negated; a far field gives a fixed state; an
// outflow repeats the face values.  Points beyond several faces resolve axis by axis: x, then
// y, then z, each in the frame of the block reached so far.
#include <cmath>
#include <cstring>

#include "cfs_internal.h"

namespace cfs {

namespace {

struct Src {
  int b, c[3];
  int flip, crossed;
  double w;
};

inline int wrapn(int i, int n) {
  int r = i % n;
  return r < 0 ? r + n : r;
}

// Lagrange basis of the nodes -1, 0, 1, 2 at t in [0, 1)
void lagrange4(double t, double* l) {
  const double tm1 = t - 1.0, tm2 = t - 2.0, tp1 = t + 1.0;
  l[0] = -(t * tm1 * tm2) / 6.0;
  l[1] = (tp1 * tm1 * tm2) / 2.0;
  l[2] = -(tp1 * t * tm2) / 2.0;
  l[3] = (tp1 * t * tm1) / 6.0;
}

// Sub-domain of block b owning point c
int owner_sid(const TopoBlock& B, const int* c) {
  int idx[3];
  for (int a = 0; a < 3; ++a) {
    const int n = B.n[a], p = B.P[a], base = n / p, rem = n % p;
    // the first rem parts have base + 1 points
    const int big = rem * (base + 1);
    idx[a] = c[a] < big ? c[a] / (base + 1) : rem + (c[a] - big) / base;
  }
  return B.sid0 + idx[0] + B.P[0] * (idx[1] + B.P[1] * idx[2]);
}

// Resolve one source through the faces; may split into up to GATHER_MAXT sources.
int resolve(const TopoBlock* B, Src* s, int n, double* cst) {
  for (int q = 0; q < n; ++q) {
    int hop = 0;
    for (; hop < 16; ++hop) {
      Src& x = s[q];
      const TopoBlock& T = B[x.b];
      int a = -1;
      for (int e = 0; e < 3; ++e)
        if (x.c[e] < 0 || x.c[e] >= T.n[e]) { a = e; break; }
      if (a < 0) break;
      const int side = x.c[a] < 0 ? 0 : 1;
      const FaceSpec& F = T.face[2 * a + side];
      switch (F.type) {
        case FACE_PERIODIC:
          x.c[a] = wrapn(x.c[a], T.n[a]);
          x.crossed = 1;
          break;
        case FACE_WALL:
          x.c[a] = side == 0 ? -x.c[a] : 2 * (T.n[a] - 1) - x.c[a];
          x.flip ^= 1;
          break;
        case FACE_OUTFLOW:
          x.c[a] = side == 0 ? 0 : T.n[a] - 1;
          break;
        case FACE_FARFIELD:
          for (int v = 0; v < 5; ++v) cst[v] += x.w * ((x.flip && v >= 1 && v <= 3) ? -F.state[v] : F.state[v]);
          s[q] = s[n - 1];
          --n;
          --q;
          hop = -1;
          break;
        case FACE_INTERFACE: {
          if (a > 1) return -1;
          const TopoBlock& T2 = B[F.nb];
          const int depth = side == 0 ? -x.c[a] : x.c[a] - (T.n[a] - 1);
          const int a2 = F.nf >> 1, s2 = F.nf & 1;
          int c2[3];
          c2[a2] = s2 == 0 ? depth - 1 : T2.n[a2] - depth;
          c2[1 - a2] = F.rev ? T.n[1 - a] - 1 - x.c[1 - a] : x.c[1 - a];
          c2[2] = x.c[2];
          x.b = F.nb;
          x.crossed = 1;
          int split = 0;
          double l[4];
          if (T2.n[2] != T.n[2]) {
            // neighbour position k nz2 / nz, floor division
            const long long num = (long long)x.c[2] * T2.n[2];
            long long k0 = num / T.n[2];
            if (k0 * T.n[2] > num) --k0;
            const long long rem = num - k0 * T.n[2];
            c2[2] = (int)k0;
            if (rem != 0) {
              split = 1;
              lagrange4((double)rem / (double)T.n[2], l);
            }
          }
          for (int e = 0; e < 3; ++e) x.c[e] = c2[e];
          if (split) {
            if (n + 3 > GATHER_MAXT) return -1;
            const Src base = x;
            for (int o = 0; o < 4; ++o) {
              Src& y = o == 0 ? s[q] : s[n + o - 1];
              y = base;
              y.c[2] = base.c[2] + o - 1;
              y.w = base.w * l[o];
            }
            n += 3;
          }
          break;
        }
        default:
          return -1;
      }
      if (hop == -1) break;  // far field: the source is gone
    }
    if (hop == 16) return -1;
  }
  return n;
}

// Coordinates at (i, j) of curvilinear block b's plane, continued across its faces: periodic
// faces wrap and add the jump, interfaces continue into the neighbour (plus the face's jump),
// physical faces reflect the grid through the boundary point, x(-m) = 2 x(0) - x(m).
bool coord(const TopoBlock* B, int b, int i, int j, int depth, double* xy) {
  if (depth > 8) return false;
  const TopoBlock& T = B[b];
  if (!T.xy) return false;
  int wrap[2] = {0, 0};
  int c[2] = {i, j};
  for (int hop = 0; hop < 4; ++hop) {
    int a = -1;
    for (int e = 0; e < 2; ++e)
      if (c[e] < 0 || c[e] >= T.n[e]) { a = e; break; }
    if (a < 0) {
      const long long n2 = (long long)T.n[0] * T.n[1];
      for (int q = 0; q < 2; ++q)
        xy[q] = T.xy[q * n2 + c[0] + (long long)T.n[0] * c[1]] + wrap[0] * T.shift[q] + wrap[1] * T.shift[2 + q];
      return true;
    }
    const int side = c[a] < 0 ? 0 : 1;
    const FaceSpec& F = T.face[2 * a + side];
    if (F.type == FACE_PERIODIC) {
      const int w = wrapn(c[a], T.n[a]);
      wrap[a] += (c[a] - w) / T.n[a];
      c[a] = w;
      continue;
    }
    double p0[2], p1[2];
    if (F.type == FACE_INTERFACE) {
      const TopoBlock& T2 = B[F.nb];
      const int d = side == 0 ? -c[a] : c[a] - (T.n[a] - 1);
      const int a2 = F.nf >> 1;
      int c2[2];
      c2[a2] = (F.nf & 1) == 0 ? d - 1 : T2.n[a2] - d;
      c2[1 - a2] = F.rev ? T.n[1 - a] - 1 - c[1 - a] : c[1 - a];
      if (!coord(B, F.nb, c2[0], c2[1], depth + 1, p0)) return false;
      for (int q = 0; q < 2; ++q) xy[q] = p0[q] + F.shift[q] + wrap[0] * T.shift[q] + wrap[1] * T.shift[2 + q];
      return true;
    }
    int cb[2] = {c[0], c[1]}, cm[2] = {c[0], c[1]};
    cb[a] = side == 0 ? 0 : T.n[a] - 1;
    cm[a] = side == 0 ? -c[a] : 2 * (T.n[a] - 1) - c[a];
    if (!coord(B, b, cb[0], cb[1], depth + 1, p0) || !coord(B, b, cm[0], cm[1], depth + 1, p1)) return false;
    for (int q = 0; q < 2; ++q) xy[q] = 2.0 * p0[q] - p1[q] + wrap[0] * T.shift[q] + wrap[1] * T.shift[2 + q];
    return true;
  }
  return false;
}

}  // namespace

bool topo_periodic(const TopoBlock& b) {
  for (int f = 0; f < 6; ++f)
    if (b.face[f].type != FACE_PERIODIC) return false;
  return true;
}

const char* topo_check(const TopoBlock* B, int nb) {
  for (int b = 0; b < nb; ++b) {
    const TopoBlock& T = B[b];
    for (int f = 0; f < 6; ++f) {
      const FaceSpec& F = T.face[f];
      if (F.type < FACE_PERIODIC || F.type > FACE_OUTFLOW) return "unknown face type";
      if (f >= 4 && F.type != FACE_PERIODIC) return "z faces must be periodic (blocks are extruded in z)";
      if (F.type != FACE_INTERFACE) continue;
      if (F.nb < 0 || F.nb >= nb || F.nf < 0 || F.nf > 3) return "interface to an unknown block or face";
      const TopoBlock& T2 = B[F.nb];
      const FaceSpec& F2 = T2.face[F.nf];
      if (F2.type != FACE_INTERFACE || F2.nb != b || F2.nf != f || F2.rev != F.rev)
        return "interface not declared the same way on both blocks";
      if (T.n[1 - (f >> 1)] != T2.n[1 - (F.nf >> 1)]) return "interface with different tangential point counts";
      if ((T.xy == nullptr) != (T2.xy == nullptr)) return "interface between a curvilinear and a Cartesian block";
      if (!T.xy && (F.nf != (f ^ 1) || F.rev)) return "Cartesian blocks join only opposite faces, unreversed";
      if ((T.n[2] == 1) != (T2.n[2] == 1)) return "interface between a 2-D and a 3-D block";
    }
  }
  return nullptr;
}

int halo_sources(const TopoBlock* B, int nb, int b, int i, int j, int k, double* out) {
  (void)nb;
  Src s[GATHER_MAXT];
  s[0].b = b;
  s[0].c[0] = i; s[0].c[1] = j; s[0].c[2] = k;
  s[0].flip = 0; s[0].crossed = 0; s[0].w = 1.0;
  double cst[5] = {0, 0, 0, 0, 0};
  const int n = resolve(B, s, 1, cst);
  if (n < 0) return -1;
  out[0] = n;
  for (int v = 0; v < 5; ++v) out[1 + v] = cst[v];
  for (int t = 0; t < GATHER_MAXT; ++t) {
    double* o = out + 6 + 7 * t;
    if (t >= n) {
      for (int q = 0; q < 7; ++q) o[q] = 0.0;
      continue;
    }
    o[0] = s[t].b; o[1] = s[t].c[0]; o[2] = s[t].c[1]; o[3] = s[t].c[2];
    o[4] = s[t].w; o[5] = s[t].flip; o[6] = s[t].crossed;
  }
  return n;
}

bool gather_entry(const TopoBlock* B, int nb, int b, int i, int j, int k, GatherEntry* e) {
  (void)nb;
  Src s[GATHER_MAXT];
  s[0].b = b;
  s[0].c[0] = i; s[0].c[1] = j; s[0].c[2] = k;
  s[0].flip = 0; s[0].crossed = 0; s[0].w = 1.0;
  std::memset(e, 0, sizeof(*e));
  const int n = resolve(B, s, 1, e->cst);
  if (n < 0) return false;
  e->nt = n;
  for (int t = 0; t < n; ++t) {
    const TopoBlock& T = B[s[t].b];
    e->off[t] = T.base + s[t].c[0] + (long long)T.n[0] * (s[t].c[1] + (long long)T.n[1] * s[t].c[2]);
    e->bN[t] = (int)T.N;
    e->sid[t] = owner_sid(T, s[t].c);
    e->w[t] = s[t].w;
    e->flags[t] = (s[t].flip ? 1 : 0) | (s[t].crossed ? 2 : 0);
  }
  return true;
}

// Metric terms (App. A) of a curvilinear block extruded in z (unit depth in 2-D): coordinate
// derivatives by the block's CD scheme in index space (Eq. 2, alpha = 0, spacing 1); the metric
// terms are the cofactors of the Jacobian matrix d(x, y, z)/d(i, j, k):
//   xi^_x = y_j z_k, xi^_y = -x_j z_k, eta^_x = -y_i z_k, eta^_y = x_i z_k,
//   zeta^_z = x_i y_j - x_j y_i, J^-1 = z_k (x_i y_j - x_j y_i), J = 1 / J^-1,
// on the (x, y) plane extended by G: beyond a periodic face the wrapped point's values, beyond
// another face the values of the continued grid to the stencil radius r (NaN deeper, where no
// flux is evaluated).
bool metric_plane(const TopoBlock* B, int nb, int b, int G, int r, int order, double dz, int ndim, double* M) {
  (void)nb;
  const TopoBlock& T = B[b];
  const int mx = T.n[0] + 2 * G, my = T.n[1] + 2 * G;
  const long long pl = (long long)mx * my;
  const double wgt[2] = {order == 4 ? 2.0 / 3.0 : 0.5, order == 4 ? -1.0 / 12.0 : 0.0};  // a/2, b/4
  const double zk = ndim == 3 ? dz : 1.0;
  for (int jj = -G; jj < T.n[1] + G; ++jj)
    for (int ii = -G; ii < T.n[0] + G; ++ii) {
      // a point beyond a periodic face takes the values of the point it wraps to
      int i = ii, j = jj;
      if ((i < 0 && T.face[0].type == FACE_PERIODIC) || (i >= T.n[0] && T.face[1].type == FACE_PERIODIC)) i = wrapn(i, T.n[0]);
      if ((j < 0 && T.face[2].type == FACE_PERIODIC) || (j >= T.n[1] && T.face[3].type == FACE_PERIODIC)) j = wrapn(j, T.n[1]);
      const int di = i < 0 ? -i : (i >= T.n[0] ? i - T.n[0] + 1 : 0);
      const int dj = j < 0 ? -j : (j >= T.n[1] ? j - T.n[1] + 1 : 0);
      double m[NMETRIC];
      bool ok = di <= r && dj <= r;
      if (ok) {
        double d[2][2] = {{0, 0}, {0, 0}};  // d[c][axis]: d x_c / d index_axis
        for (int o = 1; o <= (order == 4 ? 2 : 1) && ok; ++o) {
          double xp[2], xm[2], yp[2], ym[2];
          ok = coord(B, b, i + o, j, 0, xp) && coord(B, b, i - o, j, 0, xm) && coord(B, b, i, j + o, 0, yp) &&
               coord(B, b, i, j - o, 0, ym);
          if (!ok) break;
          for (int c = 0; c < 2; ++c) {
            d[c][0] += wgt[o - 1] * (xp[c] - xm[c]);
            d[c][1] += wgt[o - 1] * (yp[c] - ym[c]);
          }
        }
        if (ok) {
          const double det = d[0][0] * d[1][1] - d[0][1] * d[1][0];
          const double mm[NMETRIC] = {d[1][1] * zk, -d[0][1] * zk, -d[1][0] * zk, d[0][0] * zk, det, zk * det,
                                      1.0 / (zk * det)};
          for (int q = 0; q < NMETRIC; ++q) m[q] = mm[q];
          const bool inside = di == 0 && dj == 0;
          if (inside && !(det * zk > 0.0)) return false;
        }
      }
      if (!ok)
        for (int q = 0; q < NMETRIC; ++q) m[q] = NAN;
      const long long at = (long long)(ii + G) + (long long)mx * (jj + G);
      for (int q = 0; q < NMETRIC; ++q) M[q * pl + at] = m[q];
    }
  return true;
}

}  // namespace cfs
