/*
 * cfs_oracle.c -- plain, slow, FP64 CPU reference ("oracle") of the asynchronous compressible
 * flow solver hot path of arXiv 2506.03027 (Arumugam, Goswami, Vadlamani, Aditya).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this code: only the tests,
 * the smoke check and the CPU-baseline leg of the benchmark load it.  It shares no code, header,
 * table or constant generator with the CUDA library; the two meet only through seeded inputs.
 *
 * What it computes (in the paper's order):
 *   - Eq. 1 / App. A: compressible Navier-Stokes right-hand side, inviscid fluxes Eq. A2,
 *     viscous fluxes Eq. A3-A4, on a uniform Cartesian periodic grid (metric terms reduce to
 *     1/dx) or on a periodic curvilinear grid x(xi, eta), y(xi, eta), z = zeta dz given by its
 *     point coordinates: strong conservation form Eq. A1 with the metric terms xi^_x = J^-1
 *     dxi/dx (cofactors of the coordinate derivatives, by the same CD scheme in index space) and
 *     the contravariant velocities of Eq. A2.
 *   - Eq. 2 / App. B: explicit central differences CD2 (a=1,b=0) and CD4 (a=4/3,b=-1/3).
 *   - Eq. 3 / Table 4: 2N-storage low-storage RK (LSERK2, LSERK4).
 *   - Sec. 3.1, Eq. 14-15: stage-0 buffer extrapolation from delayed levels (printed polynomials).
 *   - Eq. 8 + App. C (Table 5): AT buffer updates at intermediate stages with the printed
 *     temporal-derivative polynomials; nu_j^e from Eq. 10.
 *   - Sec. 2: tenth-order Pade filter (coefficient alpha_f), applied once per step.
 *   - Alg. 1-3: SA / CAA / SAA; delays are explicit inputs, first C steps synchronous.
 *
 * Readings where the paper is silent (all documented in the design notes of the repository):
 *   - AT on nonlinear fluxes: the halo state is extrapolated / buffer-updated, fluxes are then
 *     evaluated from it (equal to c^T Phi of Eq. 7 for linear fluxes).
 *   - Halo depth: faces 2r (viscous) or r (Euler); viscous edges r x r; edge delay = max of
 *     the two faces.  Every sub-domain face is a PE boundary (also periodic self-neighbours).
 *   - Heat-flux term of Eq. A4 carries no second 1/Re (single 1/Re outside, Eq. 1).
 *   - Filter: per sub-domain line, Dirichlet closure (filtered := unfiltered at the first halo
 *     point), 11-point right side with 5 halo points, passes x -> y -> z once per step after
 *     the last stage.  Filter halo: SA = current neighbour values, AT = extrapolation with
 *     c(k+1) from the visible levels, AS = the latest visible level.
 *   - Delays: k clamped to n - C + 1 so every referenced level exists; steps n < C are SA.
 *   - CAA delay k(n) = (n - C) mod L for n >= C.
 *
 * Layout: global state U[5][nz][ny][nx] (structure of arrays, FP64), periodic in all directions.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NV 5

typedef struct {
  int nx, ny, nz;        /* global grid; nz == 1 means two-dimensional */
  int px, py, pz;        /* sub-domains per axis */
  double dx, dy, dz;     /* grid spacing */
  double gamma, mach, re, pr;
  int viscous;           /* 0: Euler, 1: Navier-Stokes */
  int visc_law;          /* 0: mu = 1, 1: mu = T^visc_exp */
  double visc_exp;
  int order;             /* 4: LSERK4-CD4-AT4 (C = 5), 2: LSERK2-CD2-AT2 (C = 3) */
  int algo;              /* 0: SA, 1: CAA, 2: SAA */
  int at;                /* 1: AT schemes, 0: AS (standard stencils on latest delayed level) */
  int caa_L;             /* CAA maximum allowable delay L */
  int kmax;              /* SAA: largest delay in the table */
  int filter;            /* 1: tenth-order Pade filter once per step */
  double alpha_f;
  double dt;
  const float* mlp;          /* learned halo network parameters (NULL: plain AT) */
  const double* mlp_scales;  /* in_scale[5], own_scale[5], out_scale[5] */
  /* curvilinear grid (NULL: uniform Cartesian): point coordinates x, y as [2][ny][nx] of a
   * mapping of (xi, eta) extruded along z (z = k dz); shift[0..1] = (x, y) jump across the
   * periodic wrap in xi, shift[2..3] = the jump across the wrap in eta */
  const double* grid_xy;
  double grid_shift[4];
} or_params;

/* ---------------------------------------------------------------- coefficient tables */

/* Table 4 (LSERK4, 8 printed digits) and App. B (LSERK2). */
int or_lserk(int order, double* A, double* B) {
  if (order == 4) {
    const double a[5] = {0.0, -0.4812317, -1.0495626, -1.6025296, -1.7782672};
    const double b[5] = {0.09761835, 0.41225329, 0.44021696, 1.42631146, 0.19787605};
    for (int i = 0; i < 5; ++i) { A[i] = a[i]; B[i] = b[i]; }
    return 5;
  }
  A[0] = 0.0; A[1] = -0.5;
  B[0] = 0.5; B[1] = 1.0;
  return 2;
}

/* Number of delayed time levels C used by the AT schemes (Sec. 3.1: 3 for AT2, 5 for AT4). */
static int or_levels(int order) { return order == 4 ? 5 : 3; }

/* Eq. 14 (order 2) and Eq. 15 (order 4): stage-0 extrapolation weights for levels
 * n-k, n-k-1, ...; the same vector is the AT spatial weight c~(k) of Eq. 7. */
void or_extrap_weights(int order, double k, double* c) {
  if (order == 2) {
    c[0] = 0.5 * (k * k + 3.0 * k + 2.0);
    c[1] = -(k * k + 2.0 * k);
    c[2] = 0.5 * (k * k + k);
    return;
  }
  double k2 = k * k, k3 = k2 * k, k4 = k3 * k;
  c[0] = (k4 + 10.0 * k3 + 35.0 * k2 + 50.0 * k + 24.0) / 24.0;
  /* Eq. 7 and Eq. 15 print 25 k^2 in this entry; the constraints of Eq. 6 (weights summing to
   * one, i.e. exact for constants) and the fourth-order extrapolation both require
   * k (k+2)(k+3)(k+4) = k^4 + 9k^3 + 26k^2 + 24k.  The printed 25 is read as a typo. */
  c[1] = -(k4 + 9.0 * k3 + 26.0 * k2 + 24.0 * k) / 6.0;
  c[2] = (k4 + 8.0 * k3 + 19.0 * k2 + 12.0 * k) / 4.0;
  c[3] = -(k4 + 7.0 * k3 + 14.0 * k2 + 8.0 * k) / 6.0;
  c[4] = (k4 + 6.0 * k3 + 11.0 * k2 + 6.0 * k) / 24.0;
}

/* Eq. 10: nu_j^e = coefficient of dt^j d^j/dt^j in the e-stage LSERK expansion; for the linear
 * test equation phi' = lambda phi this is the coefficient of z^j (z = lambda dt) of the stage
 * polynomial P_e(z), built by running the LSERK recursion of Eq. 3 on polynomials. */
double or_nu(int order, int e, int j) {
  double A[5], B[5];
  or_lserk(order, A, B);
  double P[8] = {1.0, 0, 0, 0, 0, 0, 0, 0}; /* U^(0) = 1 */
  double Q[8] = {0};
  for (int m = 0; m < e; ++m) {
    double Qn[8] = {0};
    for (int p = 0; p < 8; ++p) Qn[p] = A[m] * Q[p];
    for (int p = 0; p < 7; ++p) Qn[p + 1] += P[p]; /* + z * U^(m-1) */
    for (int p = 0; p < 8; ++p) { Q[p] = Qn[p]; P[p] += B[m] * Q[p]; }
  }
  return (j >= 0 && j < 8) ? P[j] : 0.0;
}

/* App. C: temporal derivative at a buffer point at stage e, dt * dphi/dt|^(e) = sum_l d_l phi^{n-k-l}.
 * order 2: the printed LSERK2-AT2 expression (e = 0 only); order 4: Table 5 (e = 0..3). */
void or_buffer_dudt(int order, int e, double k, double* d) {
  if (order == 2) {
    d[0] = (2.0 * k + 3.0) / 2.0;
    d[1] = -(2.0 * k + 2.0);
    d[2] = (2.0 * k + 1.0) / 2.0;
    return;
  }
  double n1 = e >= 1 ? or_nu(4, e, 1) : 0.0;
  double n2 = e >= 2 ? or_nu(4, e, 2) : 0.0;
  double n3 = e >= 3 ? or_nu(4, e, 3) : 0.0;
  double k2 = k * k, k3 = k2 * k;
  d[0] = (2 * k3 + (15 + 6 * n1) * k2 + (35 + 30 * n1 + 12 * n2) * k + 25 + 35 * n1 + 30 * n2 + 12 * n3) / 12.0;
  d[1] = -(4 * k3 + (27 + 12 * n1) * k2 + (52 + 54 * n1 + 24 * n2) * k + 24 + 52 * n1 + 54 * n2 + 24 * n3) / 6.0;
  d[2] = (2 * k3 + (12 + 6 * n1) * k2 + (19 + 24 * n1 + 12 * n2) * k + 6 + 19 * n1 + 24 * n2 + 12 * n3) / 2.0;
  d[3] = -(4 * k3 + (21 + 12 * n1) * k2 + (28 + 42 * n1 + 24 * n2) * k + 8 + 28 * n1 + 42 * n2 + 24 * n3) / 6.0;
  d[4] = (2 * k3 + (9 + 6 * n1) * k2 + (11 + 18 * n1 + 12 * n2) * k + 3 + 11 * n1 + 18 * n2 + 12 * n3) / 12.0;
}

/* Tenth-order Pade filter (Sec. 2, after Visbal & Gaitonde 2002): right-side coefficients a_0..a_5
 * of  alpha f^_{i-1} + f^_i + alpha f^_{i+1} = sum_n (a_n / 2)(f_{i+n} + f_{i-n}). */
void or_filter_coeffs(double al, double* a) {
  a[0] = (193.0 + 126.0 * al) / 256.0;
  a[1] = (105.0 + 302.0 * al) / 256.0;
  a[2] = 15.0 * (-1.0 + 2.0 * al) / 64.0;
  a[3] = 45.0 * (1.0 - 2.0 * al) / 512.0;
  a[4] = 5.0 * (-1.0 + 2.0 * al) / 256.0;
  a[5] = (1.0 - 2.0 * al) / 512.0;
}

/* Filter one line: n interior values f[5..5+n), 5 halo values on each side (f has n + 10 entries).
 * Dirichlet closure: the filtered value at the first halo point equals its unfiltered value.
 * Tridiagonal system solved by plain Gaussian elimination without pivoting (Thomas). */
void or_filter_line(int n, double al, const double* f, double* out) {
  double a[6];
  or_filter_coeffs(al, a);
  double* rhs = (double*)malloc(sizeof(double) * n);
  double* cp = (double*)malloc(sizeof(double) * n);
  for (int i = 0; i < n; ++i) {
    const double* c = f + 5 + i;
    double s = a[0] * c[0];
    for (int m = 1; m <= 5; ++m) s += 0.5 * a[m] * (c[m] + c[-m]);
    rhs[i] = s;
  }
  rhs[0] -= al * f[4];          /* known filtered value at the first left halo point */
  rhs[n - 1] -= al * f[5 + n];  /* ... and at the first right halo point */
  /* forward sweep: diag 1, off-diagonals al */
  double diag = 1.0;
  cp[0] = al / diag;
  rhs[0] = rhs[0] / diag;
  for (int i = 1; i < n; ++i) {
    double m = 1.0 - al * cp[i - 1];
    cp[i] = al / m;
    rhs[i] = (rhs[i] - al * rhs[i - 1]) / m;
  }
  out[n - 1] = rhs[n - 1];
  for (int i = n - 2; i >= 0; --i) out[i] = rhs[i] - cp[i] * out[i + 1];
  free(rhs);
  free(cp);
}

/* ---------------------------------------------------------------- decomposition helpers */

/* Split n points into p parts as evenly as possible; the first n % p parts get one extra. */
static void split_axis(int n, int p, int idx, int* off, int* len) {
  int base = n / p, rem = n % p;
  *len = base + (idx < rem ? 1 : 0);
  *off = idx * base + (idx < rem ? idx : rem);
}

static inline int wrapi(int i, int n) {
  int r = i % n;
  return r < 0 ? r + n : r;
}

typedef struct {
  int ox, oy, oz, sx, sy, sz;  /* owned box */
  int g, gz;                   /* ghost depth in x/y and in z (0 in 2-D) */
  int ex, ey, ez;              /* extended dims */
} subdom;

static void make_subdom(const or_params* p, int s, int g, subdom* d) {
  int nsx = p->px, nsy = p->py;
  int ix = s % nsx, iy = (s / nsx) % nsy, iz = s / (nsx * nsy);
  split_axis(p->nx, p->px, ix, &d->ox, &d->sx);
  split_axis(p->ny, p->py, iy, &d->oy, &d->sy);
  split_axis(p->nz, p->pz, iz, &d->oz, &d->sz);
  d->g = g;
  d->gz = (p->nz > 1) ? g : 0;
  d->ex = d->sx + 2 * g;
  d->ey = d->sy + 2 * g;
  d->ez = d->sz + 2 * d->gz;
}

/* Classify extended point (i,j,k): returns number of coordinates outside the owned box and fills
 * depth per axis (0 inside) and the face index (0..5: -x,+x,-y,+y,-z,+z) of each outside axis. */
static int classify(const subdom* d, int i, int j, int k, int dep[3], int face[3]) {
  int c[3] = {i - d->g, j - d->g, k - d->gz};
  int s[3] = {d->sx, d->sy, d->sz};
  int nout = 0;
  for (int a = 0; a < 3; ++a) {
    dep[a] = 0;
    face[a] = -1;
    if (c[a] < 0) { dep[a] = -c[a]; face[a] = 2 * a; nout++; }
    else if (c[a] >= s[a]) { dep[a] = c[a] - s[a] + 1; face[a] = 2 * a + 1; nout++; }
  }
  return nout;
}

/* ---------------------------------------------------------------- metric terms (curvilinear)
 * For the extruded mapping the Jacobian matrix d(x,y,z)/d(xi,eta,zeta) is
 * [[x_xi, x_eta, 0], [y_xi, y_eta, 0], [0, 0, z_zeta]] with z_zeta = dz (1 in 2-D); its
 * cofactors are the metric terms of App. A:
 *   xi^_x = y_eta z_zeta, xi^_y = -x_eta z_zeta, eta^_x = -y_xi z_zeta, eta^_y = x_xi z_zeta,
 *   zeta^_z = x_xi y_eta - x_eta y_xi,  J^-1 = z_zeta (x_xi y_eta - x_eta y_xi),
 * all other metric terms zero.  The coordinate derivatives use the scheme of Eq. 2 in index
 * space (spacing 1), periodic with the coordinate jump added across the wrap.  With periodic CD
 * operators D_xi D_eta = D_eta D_xi, so sum_a D_a (metric column) = 0 holds discretely and a
 * uniform flow stays uniform (freestream preservation). */
#define NM 6 /* xi^_x, xi^_y, eta^_x, eta^_y, zeta^_z, J^-1 */

static double coord_at(const or_params* p, int c, int i, int j) {
  int ii = wrapi(i, p->nx), jj = wrapi(j, p->ny);
  int wi = (i - ii) / p->nx, wj = (j - jj) / p->ny; /* number of wraps (exact multiples) */
  return p->grid_xy[(size_t)c * p->nx * p->ny + (size_t)ii + (size_t)p->nx * jj] + wi * p->grid_shift[c] +
         wj * p->grid_shift[2 + c];
}

static double cd_coord(const or_params* p, int c, int i, int j, int axis) {
  double f[5];
  for (int o = -2; o <= 2; ++o) f[o + 2] = axis == 0 ? coord_at(p, c, i + o, j) : coord_at(p, c, i, j + o);
  if (p->order == 4) return (-1.0 / 3.0) * (f[4] - f[0]) / 4.0 + (4.0 / 3.0) * (f[3] - f[1]) / 2.0;
  return (f[3] - f[1]) / 2.0;
}

/* Metric field [NM][N] of the whole grid (NULL for a Cartesian grid). */
static double* metric_field(const or_params* p) {
  if (!p->grid_xy) return NULL;
  const size_t N = (size_t)p->nx * p->ny * p->nz, n2 = (size_t)p->nx * p->ny;
  double* M = (double*)malloc(sizeof(double) * NM * N);
  const double zz = p->nz > 1 ? p->dz : 1.0;
  for (int j = 0; j < p->ny; ++j)
    for (int i = 0; i < p->nx; ++i) {
      double x_xi = cd_coord(p, 0, i, j, 0), x_eta = cd_coord(p, 0, i, j, 1);
      double y_xi = cd_coord(p, 1, i, j, 0), y_eta = cd_coord(p, 1, i, j, 1);
      double det = x_xi * y_eta - x_eta * y_xi;
      double m[NM] = {y_eta * zz, -x_eta * zz, -y_xi * zz, x_xi * zz, det, zz * det};
      for (int k = 0; k < p->nz; ++k)
        for (int c = 0; c < NM; ++c) M[(size_t)c * N + (size_t)i + (size_t)p->nx * j + n2 * k] = m[c];
    }
  return M;
}

/* ---------------------------------------------------------------- RHS on an extended array */

typedef struct {
  double* E;     /* [5][ext] conserved values (NaN where not filled) */
  double* W;     /* [7][ext] rho,u,v,w,p,T,mu */
  double* G;     /* [12][ext] du/dx.. (u,v,w,T) x (x,y,z) */
  double* F;     /* [3][5][ext] inviscid fluxes per direction */
  double* FV;    /* [3][5][ext] viscous fluxes per direction */
  double* M;     /* [NM][ext] metric terms (curvilinear grids) */
  size_t cap;
} work_t;

static void work_reserve(work_t* w, size_t n) {
  if (w->cap >= n) return;
  free(w->E); free(w->W); free(w->G); free(w->F); free(w->FV); free(w->M);
  w->M = (double*)malloc(sizeof(double) * NM * n);
  w->E = (double*)malloc(sizeof(double) * NV * n);
  w->W = (double*)malloc(sizeof(double) * 7 * n);
  w->G = (double*)malloc(sizeof(double) * 12 * n);
  w->F = (double*)malloc(sizeof(double) * 15 * n);
  w->FV = (double*)malloc(sizeof(double) * 15 * n);
  w->cap = n;
}

static void work_free(work_t* w) {
  free(w->E); free(w->W); free(w->G); free(w->F); free(w->FV); free(w->M);
  memset(w, 0, sizeof(*w));
}

/* Eq. 2 with alpha = 0: derivative at index i of samples spaced by `st`, spacing h. */
static inline double cd(const double* f, size_t i, size_t st, int order, double h) {
  if (order == 4) {
    const double a = 4.0 / 3.0, b = -1.0 / 3.0;
    return (b * (f[i + 2 * st] - f[i - 2 * st]) / 4.0 + a * (f[i + st] - f[i - st]) / 2.0) / h;
  }
  return (f[i + st] - f[i - st]) / (2.0 * h);
}

/* Right-hand side R(U) at the owned points of sub-domain d, from the filled extended array E.
 * Output R[5][sz][sy][sx]. */
static void rhs_ext(const or_params* p, const subdom* d, work_t* w, double* R) {
  const size_t ex = d->ex, ey = d->ey, ez = d->ez;
  const size_t n = ex * ey * ez;
  const size_t sty = ex, stz = ex * ey;
  const int three_d = p->nz > 1;
  const double gm = p->gamma, M2 = p->mach * p->mach;
  const int r = (p->order == 4) ? 2 : 1;
  double* E = w->E;
  double* W = w->W;
  /* primitives (App. A: E_t = T/(gamma(gamma-1)M^2) + |u|^2/2, p = rho T/(gamma M^2)) */
  for (size_t q = 0; q < n; ++q) {
    double rho = E[q], ru = E[n + q], rv = E[2 * n + q], rw = E[3 * n + q], rE = E[4 * n + q];
    double u = ru / rho, v = rv / rho, ww = rw / rho;
    double pr = (gm - 1.0) * (rE - 0.5 * rho * (u * u + v * v + ww * ww));
    double T = gm * M2 * pr / rho;
    W[q] = rho; W[n + q] = u; W[2 * n + q] = v; W[3 * n + q] = ww; W[4 * n + q] = pr; W[5 * n + q] = T;
    W[6 * n + q] = (p->visc_law == 1) ? pow(T, p->visc_exp) : 1.0;
  }
  const double h[3] = {p->dx, p->dy, p->dz};
  const size_t st[3] = {1, sty, stz};
  const int ndim = three_d ? 3 : 2;
  const int lo[3] = {r, r, three_d ? r : 0};
  const int hi[3] = {(int)ex - r, (int)ey - r, three_d ? (int)ez - r : 1};
  /* inviscid fluxes Eq. A2 (Cartesian: xi_x = 1) at every extended point */
  for (int a = 0; a < ndim; ++a) {
    double* F = w->F + (size_t)a * NV * n;
    for (size_t q = 0; q < n; ++q) {
      double rho = W[q], ua = W[(1 + a) * n + q], pr = W[4 * n + q];
      F[q] = rho * ua;
      F[n + q] = rho * W[n + q] * ua + (a == 0 ? pr : 0.0);
      F[2 * n + q] = rho * W[2 * n + q] * ua + (a == 1 ? pr : 0.0);
      F[3 * n + q] = rho * W[3 * n + q] * ua + (a == 2 ? pr : 0.0);
      F[4 * n + q] = (E[4 * n + q] + pr) * ua;
    }
  }
  if (p->viscous) {
    /* gradients of u, v, w, T at points where the CD stencil fits inside the extended array */
    double* G = w->G;
    for (size_t q = 0; q < 12 * n; ++q) G[q] = NAN;
    for (int k = lo[2]; k < hi[2]; ++k)
      for (int j = r; j < (int)ey - r; ++j)
        for (int i = r; i < (int)ex - r; ++i) {
          size_t q = (size_t)i + sty * j + stz * k;
          for (int vv = 0; vv < 4; ++vv) {
            const double* f = W + (size_t)(vv == 3 ? 5 : 1 + vv) * n;
            for (int a = 0; a < 3; ++a)
              G[(size_t)(3 * vv + a) * n + q] = (a < ndim) ? cd(f, q, st[a], p->order, h[a]) : 0.0;
          }
        }
    /* viscous fluxes Eq. A3-A4: F_v,a = [0, tau_a1, tau_a2, tau_a3, u_j tau_aj + kappa dT/dx_a] */
    const double kap = 1.0 / ((gm - 1.0) * p->pr * M2);
    for (size_t q = 0; q < n; ++q) {
      double mu = W[6 * n + q];
      double du[3][3];  /* du[i][j] = d u_i / d x_j */
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) du[i][j] = G[(size_t)(3 * i + j) * n + q];
      double div = du[0][0] + du[1][1] + du[2][2];
      double tau[3][3];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
          tau[i][j] = mu * (du[i][j] + du[j][i]) - (i == j ? 2.0 / 3.0 * mu * div : 0.0);
      double uu[3] = {W[n + q], W[2 * n + q], W[3 * n + q]};
      for (int a = 0; a < ndim; ++a) {
        double* FV = w->FV + (size_t)a * NV * n;
        FV[q] = 0.0;
        FV[n + q] = tau[a][0];
        FV[2 * n + q] = tau[a][1];
        FV[3 * n + q] = tau[a][2];
        FV[4 * n + q] = uu[0] * tau[a][0] + uu[1] * tau[a][1] + uu[2] * tau[a][2] +
                        kap * mu * G[(size_t)(9 + a) * n + q];
      }
    }
  }
  /* Eq. 1 on a uniform Cartesian grid: R = -sum_a D_a F_a + (1/Re) sum_a D_a Fv_a */
  const double ire = 1.0 / p->re;
  for (int k = 0; k < d->sz; ++k)
    for (int j = 0; j < d->sy; ++j)
      for (int i = 0; i < d->sx; ++i) {
        size_t q = (size_t)(i + d->g) + sty * (j + d->g) + stz * (k + d->gz);
        size_t o = (size_t)i + (size_t)d->sx * (j + (size_t)d->sy * k);
        size_t no = (size_t)d->sx * d->sy * d->sz;
        for (int vv = 0; vv < NV; ++vv) {
          double acc = 0.0;
          for (int a = 0; a < ndim; ++a) {
            const double* F = w->F + (size_t)a * NV * n + (size_t)vv * n;
            acc -= cd(F, q, st[a], p->order, h[a]);
            if (p->viscous) {
              const double* FV = w->FV + (size_t)a * NV * n + (size_t)vv * n;
              acc += ire * cd(FV, q, st[a], p->order, h[a]);
            }
          }
          R[vv * no + o] = acc;
        }
      }
}

/* Curvilinear right-hand side (Eq. A1 with a time-invariant grid): at the owned points
 *   dU/dt = J [ -sum_a D_a F^_a + (1/Re) sum_a D_a F^v_a ],
 * D_a the scheme of Eq. 2 along index direction a (spacing 1), F^_a of Eq. A2 with the
 * contravariant velocity U^_a = (metric row a) . u, F^v_a of Eq. A3 = (metric row a) . (Fv_x, Fv_y,
 * Fv_z), and the stresses / heat flux of Eq. A4 from physical gradients
 * d phi / d x_j = J sum_k (metric row k)_j d phi / d xi_k.  Mg: global metric field [NM][N]. */
static void rhs_ext_curv(const or_params* p, const subdom* d, const double* Mg, work_t* w, double* R) {
  const size_t ex = d->ex, ey = d->ey, ez = d->ez;
  const size_t n = ex * ey * ez;
  const size_t N = (size_t)p->nx * p->ny * p->nz;
  const size_t sty = ex, stz = ex * ey;
  const int three_d = p->nz > 1;
  const int ndim = three_d ? 3 : 2;
  const double gm = p->gamma, M2 = p->mach * p->mach;
  const int r = (p->order == 4) ? 2 : 1;
  double* E = w->E;
  double* W = w->W;
  double* Mx = w->M;
  /* metric terms at every extended point (periodic) */
  for (int k = 0; k < (int)ez; ++k)
    for (int j = 0; j < (int)ey; ++j)
      for (int i = 0; i < (int)ex; ++i) {
        int gx = wrapi(d->ox + i - d->g, p->nx), gy = wrapi(d->oy + j - d->g, p->ny);
        int gz = wrapi(d->oz + k - d->gz, p->nz);
        size_t gq = (size_t)gx + (size_t)p->nx * (gy + (size_t)p->ny * gz);
        size_t q = (size_t)i + ex * (j + ey * (size_t)k);
        for (int c = 0; c < NM; ++c) Mx[c * n + q] = Mg[c * N + gq];
      }
  /* metric row of index direction a at point q: (d xi_a / d x, d xi_a / d y, d xi_a / d z) / J */
#define MROW(a, q, out)                                                             \
  do {                                                                              \
    if ((a) == 0) { out[0] = Mx[q]; out[1] = Mx[n + (q)]; out[2] = 0.0; }           \
    else if ((a) == 1) { out[0] = Mx[2 * n + (q)]; out[1] = Mx[3 * n + (q)]; out[2] = 0.0; } \
    else { out[0] = 0.0; out[1] = 0.0; out[2] = Mx[4 * n + (q)]; }                  \
  } while (0)
  for (size_t q = 0; q < n; ++q) {
    double rho = E[q], ru = E[n + q], rv = E[2 * n + q], rw = E[3 * n + q], rE = E[4 * n + q];
    double u = ru / rho, v = rv / rho, ww = rw / rho;
    double pr = (gm - 1.0) * (rE - 0.5 * rho * (u * u + v * v + ww * ww));
    double T = gm * M2 * pr / rho;
    W[q] = rho; W[n + q] = u; W[2 * n + q] = v; W[3 * n + q] = ww; W[4 * n + q] = pr; W[5 * n + q] = T;
    W[6 * n + q] = (p->visc_law == 1) ? pow(T, p->visc_exp) : 1.0;
  }
  const size_t st[3] = {1, sty, stz};
  const int lo2 = three_d ? r : 0, hi2 = three_d ? (int)ez - r : 1;
  /* Eq. A2: F^_a = [rho U^, rho u U^ + m_x p, rho v U^ + m_y p, rho w U^ + m_z p, (rho E_t + p) U^] */
  for (int a = 0; a < ndim; ++a) {
    double* F = w->F + (size_t)a * NV * n;
    for (size_t q = 0; q < n; ++q) {
      double m[3];
      MROW(a, q, m);
      double rho = W[q], pr = W[4 * n + q];
      double Uc = m[0] * W[n + q] + m[1] * W[2 * n + q] + m[2] * W[3 * n + q];
      F[q] = rho * Uc;
      F[n + q] = rho * W[n + q] * Uc + m[0] * pr;
      F[2 * n + q] = rho * W[2 * n + q] * Uc + m[1] * pr;
      F[3 * n + q] = rho * W[3 * n + q] * Uc + m[2] * pr;
      F[4 * n + q] = (E[4 * n + q] + pr) * Uc;
    }
  }
  if (p->viscous) {
    double* G = w->G;
    for (size_t q = 0; q < 12 * n; ++q) G[q] = NAN;
    for (int k = lo2; k < hi2; ++k)
      for (int j = r; j < (int)ey - r; ++j)
        for (int i = r; i < (int)ex - r; ++i) {
          size_t q = (size_t)i + sty * j + stz * k;
          double J = 1.0 / Mx[5 * n + q];
          for (int vv = 0; vv < 4; ++vv) {
            const double* f = W + (size_t)(vv == 3 ? 5 : 1 + vv) * n;
            double dxi[3];
            for (int a = 0; a < 3; ++a) dxi[a] = (a < ndim) ? cd(f, q, st[a], p->order, 1.0) : 0.0;
            for (int jj = 0; jj < 3; ++jj) {
              double acc = 0.0;
              for (int a = 0; a < ndim; ++a) {
                double m[3];
                MROW(a, q, m);
                acc += m[jj] * dxi[a];
              }
              G[(size_t)(3 * vv + jj) * n + q] = J * acc;
            }
          }
        }
    const double kap = 1.0 / ((gm - 1.0) * p->pr * M2);
    for (size_t q = 0; q < n; ++q) {
      double mu = W[6 * n + q];
      double du[3][3];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) du[i][j] = G[(size_t)(3 * i + j) * n + q];
      double div = du[0][0] + du[1][1] + du[2][2];
      double tau[3][3], b[3];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
          tau[i][j] = mu * (du[i][j] + du[j][i]) - (i == j ? 2.0 / 3.0 * mu * div : 0.0);
      double uu[3] = {W[n + q], W[2 * n + q], W[3 * n + q]};
      for (int i = 0; i < 3; ++i)
        b[i] = uu[0] * tau[i][0] + uu[1] * tau[i][1] + uu[2] * tau[i][2] + kap * mu * G[(size_t)(9 + i) * n + q];
      /* Eq. A3: F^v_a = [0, m_i tau_i1, m_i tau_i2, m_i tau_i3, m_i b_i] */
      for (int a = 0; a < ndim; ++a) {
        double m[3];
        MROW(a, q, m);
        double* FV = w->FV + (size_t)a * NV * n;
        FV[q] = 0.0;
        for (int c = 0; c < 3; ++c) FV[(1 + c) * n + q] = m[0] * tau[0][c] + m[1] * tau[1][c] + m[2] * tau[2][c];
        FV[4 * n + q] = m[0] * b[0] + m[1] * b[1] + m[2] * b[2];
      }
    }
  }
#undef MROW
  const double ire = 1.0 / p->re;
  for (int k = 0; k < d->sz; ++k)
    for (int j = 0; j < d->sy; ++j)
      for (int i = 0; i < d->sx; ++i) {
        size_t q = (size_t)(i + d->g) + sty * (j + d->g) + stz * (k + d->gz);
        size_t o = (size_t)i + (size_t)d->sx * (j + (size_t)d->sy * k);
        size_t no = (size_t)d->sx * d->sy * d->sz;
        double J = 1.0 / Mx[5 * n + q];
        for (int vv = 0; vv < NV; ++vv) {
          double acc = 0.0;
          for (int a = 0; a < ndim; ++a) {
            const double* F = w->F + (size_t)a * NV * n + (size_t)vv * n;
            acc -= cd(F, q, st[a], p->order, 1.0);
            if (p->viscous) {
              const double* FV = w->FV + (size_t)a * NV * n + (size_t)vv * n;
              acc += ire * cd(FV, q, st[a], p->order, 1.0);
            }
          }
          R[vv * no + o] = J * acc;
        }
      }
}

/* ---------------------------------------------------------------- learned halo (FP64 reference)
 * A 3-layer perceptron 65 -> 64 -> 64 -> 20 (GELU, tanh form) predicts, per face column of 4 halo
 * points, (U^n - three-level extrapolation of Eq. 14) * out_scale from features of the delayed
 * levels rounded to BF16.  Parameter layout: W1[64][65], b1[64], W2[64][64], b2[64], W3[20][64], b3[20]. */
#define OM_NIN 65
#define OM_NH 64
#define OM_NOUT 20
#define OM_DEPTH 4

/* FP64 -> FP32 (round to nearest) -> BF16 (round to nearest even), returned as a double */
double or_bf16(double x) {
  float f = (float)x;
  uint32_t b;
  memcpy(&b, &f, 4);
  b += 0x7FFFu + ((b >> 16) & 1u);
  b &= 0xFFFF0000u;
  memcpy(&f, &b, 4);
  return (double)f;
}

static double om_gelu(double z) {
  const double k0 = 0.7978845608028654, k1 = 0.044715;
  return 0.5 * z * (1.0 + tanh(k0 * (z + k1 * z * z * z)));
}

/* y = MLP(x) in FP64 with the FP32 parameters */
void or_mlp_forward(const float* P, const double* x, double* y) {
  const float* W1 = P;
  const float* b1 = W1 + OM_NH * OM_NIN;
  const float* W2 = b1 + OM_NH;
  const float* b2 = W2 + OM_NH * OM_NH;
  const float* W3 = b2 + OM_NH;
  const float* b3 = W3 + OM_NOUT * OM_NH;
  double h1[OM_NH], h2[OM_NH];
  for (int o = 0; o < OM_NH; ++o) {
    double a = b1[o];
    for (int i = 0; i < OM_NIN; ++i) a += (double)W1[o * OM_NIN + i] * x[i];
    h1[o] = om_gelu(a);
  }
  for (int o = 0; o < OM_NH; ++o) {
    double a = b2[o];
    for (int i = 0; i < OM_NH; ++i) a += (double)W2[o * OM_NH + i] * h1[i];
    h2[o] = om_gelu(a);
  }
  for (int o = 0; o < OM_NOUT; ++o) {
    double a = b3[o];
    for (int i = 0; i < OM_NH; ++i) a += (double)W3[o * OM_NH + i] * h2[i];
    y[o] = a;
  }
}

/* Global index of point j (1..4) of the column of face f at owned tangential coordinates (t1, t2):
 * the halo point at depth j outside the face (halo = 1) or the own point at depth j inside it. */
static size_t om_point(const or_params* p, const subdom* d, int f, int t1, int t2, int j, int halo) {
  int a = f / 2, side = f % 2;
  int c[3], o[3] = {d->ox, d->oy, d->oz}, sz[3] = {d->sx, d->sy, d->sz}, n[3] = {p->nx, p->ny, p->nz};
  c[(a + 1) % 3] = t1;
  c[(a + 2) % 3] = t2;
  if (halo) c[a] = side == 0 ? -j : sz[a] - 1 + j;
  else c[a] = side == 0 ? j - 1 : sz[a] - j;
  int g[3];
  for (int q = 0; q < 3; ++q) g[q] = wrapi(o[q] + c[q], n[q]);
  return (size_t)g[0] + (size_t)p->nx * (g[1] + (size_t)p->ny * g[2]);
}

/* Features (BF16-rounded) and the three-level extrapolation of one column at delay k. */
void or_column_features(const or_params* p, const double* const* lev /* [0]=U^n [1]=U^{n-k} [2]=U^{n-k-1} [3]=U^{n-k-2} */,
                        int s, int f, int t1, int t2, int k, double* x, double* at3) {
  const size_t N = (size_t)p->nx * p->ny * p->nz;
  subdom d;
  make_subdom(p, s, 0, &d);
  const double* in = p->mlp_scales;
  const double* own = p->mlp_scales + 5;
  double c3[5];
  or_extrap_weights(2, (double)k, c3);
  for (int j = 1; j <= OM_DEPTH; ++j) {
    size_t gh = om_point(p, &d, f, t1, t2, j, 1), go = om_point(p, &d, f, t1, t2, j, 0);
    for (int v = 0; v < 5; ++v) {
      double a = lev[1][v * N + gh], b = lev[2][v * N + gh], c = lev[3][v * N + gh];
      x[(j - 1) * 5 + v] = or_bf16((a - b) * in[v]);
      x[20 + (j - 1) * 5 + v] = or_bf16((b - c) * in[v]);
      x[40 + (j - 1) * 5 + v] = or_bf16((lev[0][v * N + go] - lev[1][v * N + go]) * own[v]);
      at3[(j - 1) * 5 + v] = c3[0] * a + c3[1] * b + c3[2] * c;
    }
  }
  for (int q = 0; q < 5; ++q) x[60 + q] = (q == k) ? 1.0 : 0.0;
}

/* ---------------------------------------------------------------- the time loop (Alg. 1-3) */

/* delay of face f of sub-domain s at step n before clamping */
static int raw_delay(const or_params* p, const int8_t* delays, int nsub, long n, int s, int f) {
  int C = or_levels(p->order);
  if (p->algo == 1) return (int)((n - C) % p->caa_L);           /* CAA: uniform periodic */
  if (p->algo == 2) return delays[((size_t)n * nsub + s) * 6 + f]; /* SAA: explicit table */
  return 0;
}

/* Ring of full global states indexed by time level. */
typedef struct {
  double** lev;
  int R;
} hist_t;

static inline const double* H(const hist_t* h, long level) { return h->lev[level % h->R]; }

typedef struct {
  /* per-sub-domain AT halo buffers (Eq. 8): U_buf, Q_buf at the needed foreign points */
  double* ub;
  double* qb;
  size_t cap;
} halo_t;

/* Fill the extended array of sub-domain d for stage m-1 of step n.
 * mode: 0 SA (neighbour's current values from Ucur), 1 AT (halo buffer), 2 AS (level n-k). */
static void fill_ext(const or_params* p, const subdom* d, const double* Ucur, int mode, const hist_t* h,
                     long n, const int* kf, const halo_t* hb, work_t* w) {
  const size_t ex = d->ex, ey = d->ey, ez = d->ez, ne = ex * ey * ez;
  const size_t N = (size_t)p->nx * p->ny * p->nz;
  const int r = (p->order == 4) ? 2 : 1;
  for (size_t q = 0; q < NV * ne; ++q) w->E[q] = NAN;
  for (int k = 0; k < (int)ez; ++k)
    for (int j = 0; j < (int)ey; ++j)
      for (int i = 0; i < (int)ex; ++i) {
        int dep[3], face[3];
        int nout = classify(d, i, j, k, dep, face);
        int need = 0, kd = 0;
        if (nout == 0) need = 1;
        else if (nout == 1) {
          need = 1;
          for (int a = 0; a < 3; ++a) if (face[a] >= 0) kd = kf[face[a]];
        } else if (nout == 2 && p->viscous) {
          need = 1;
          kd = 0;
          for (int a = 0; a < 3; ++a) {
            if (face[a] >= 0) {
              if (dep[a] > r) need = 0;
              if (kf[face[a]] > kd) kd = kf[face[a]];
            }
          }
        }
        if (!need) continue;
        int gx = wrapi(d->ox + i - d->g, p->nx), gy = wrapi(d->oy + j - d->g, p->ny);
        int gz = wrapi(d->oz + k - d->gz, p->nz);
        size_t gq = (size_t)gx + (size_t)p->nx * (gy + (size_t)p->ny * gz);
        size_t q = (size_t)i + ex * (j + ey * k);
        for (int v = 0; v < NV; ++v) {
          double val;
          if (nout == 0 || mode == 0) val = Ucur[v * N + gq];
          else if (mode == 1) val = hb->ub[v * ne + q];
          else val = H(h, n - kd)[v * N + gq];
          w->E[v * ne + q] = val;
        }
      }
}

/* Delay of each needed foreign extended point (face delay, or max of two faces on an edge). */
static int point_delay(const or_params* p, const subdom* d, int i, int j, int k, const int* kf, int* need) {
  int dep[3], face[3];
  int nout = classify(d, i, j, k, dep, face);
  const int r = (p->order == 4) ? 2 : 1;
  *need = 0;
  if (nout == 1) {
    *need = 1;
    for (int a = 0; a < 3; ++a) if (face[a] >= 0) return kf[face[a]];
  }
  if (nout == 2 && p->viscous) {
    int kd = 0;
    *need = 1;
    for (int a = 0; a < 3; ++a)
      if (face[a] >= 0) {
        if (dep[a] > r) *need = 0;
        if (kf[face[a]] > kd) kd = kf[face[a]];
      }
    return kd;
  }
  return 0;
}

/* AT halo buffer: stage-0 extrapolation (Eq. 14/15), then buffer updates (Eq. 8, App. C). */
static void halo_init(const or_params* p, const subdom* d, const hist_t* h, long n, const int* kf, halo_t* hb) {
  const size_t ex = d->ex, ey = d->ey, ez = d->ez, ne = ex * ey * ez;
  const size_t N = (size_t)p->nx * p->ny * p->nz;
  const int C = or_levels(p->order);
  for (int k = 0; k < (int)ez; ++k)
    for (int j = 0; j < (int)ey; ++j)
      for (int i = 0; i < (int)ex; ++i) {
        int need;
        int kd = point_delay(p, d, i, j, k, kf, &need);
        if (!need) continue;
        double c[5];
        or_extrap_weights(p->order, (double)kd, c);
        int gx = wrapi(d->ox + i - d->g, p->nx), gy = wrapi(d->oy + j - d->g, p->ny);
        int gz = wrapi(d->oz + k - d->gz, p->nz);
        size_t gq = (size_t)gx + (size_t)p->nx * (gy + (size_t)p->ny * gz);
        size_t q = (size_t)i + ex * (j + ey * k);
        for (int v = 0; v < NV; ++v) {
          double s = 0.0;
          for (int l = 0; l < C; ++l) s += c[l] * H(h, n - kd - l)[v * N + gq];
          hb->ub[v * ne + q] = s;
          hb->qb[v * ne + q] = 0.0;
        }
      }
}

/* With a learned halo model: U_buf^(0) of every face column is the extrapolation plus the
 * network's residual; Q_buf stays zero and the buffer updates of Eq. 8 proceed unchanged. */
static void halo_init_learned(const or_params* p, const subdom* d, int s, const hist_t* h, long n, const int* kf,
                              halo_t* hb) {
  const size_t ex = d->ex, ey = d->ey, ne = ex * ey * d->ez;
  const int nd = p->nz > 1 ? 3 : 2;
  const int sz[3] = {d->sx, d->sy, d->sz};
  const double* out = p->mlp_scales + 10;
  for (int f = 0; f < 2 * nd; ++f) {
    int a = f / 2, side = f % 2, b1 = (a + 1) % 3, b2 = (a + 2) % 3;
    int k = kf[f];
    const double* lev[4] = {H(h, n), H(h, n - k), H(h, n - k - 1), H(h, n - k - 2)};
    for (int t2 = 0; t2 < sz[b2]; ++t2)
      for (int t1 = 0; t1 < sz[b1]; ++t1) {
        double x[OM_NIN], at3[OM_NOUT], y[OM_NOUT];
        or_column_features(p, lev, s, f, t1, t2, k, x, at3);
        or_mlp_forward(p->mlp, x, y);
        for (int j = 1; j <= OM_DEPTH; ++j) {
          int c[3];
          c[b1] = t1;
          c[b2] = t2;
          c[a] = side == 0 ? -j : sz[a] - 1 + j;
          size_t q = (size_t)(c[0] + d->g) + ex * ((c[1] + d->g) + ey * (c[2] + d->gz));
          for (int v = 0; v < 5; ++v) {
            hb->ub[v * ne + q] = at3[(j - 1) * 5 + v] + y[(j - 1) * 5 + v] / out[v];
            hb->qb[v * ne + q] = 0.0;
          }
        }
      }
  }
}

static void halo_update(const or_params* p, const subdom* d, const hist_t* h, long n, const int* kf, int m,
                        const double* A, const double* B, halo_t* hb) {
  /* buffer update at stage m (1-based) uses the temporal derivative at stage e = m - 1 */
  const size_t ex = d->ex, ey = d->ey, ez = d->ez, ne = ex * ey * ez;
  const size_t N = (size_t)p->nx * p->ny * p->nz;
  const int C = or_levels(p->order);
  for (int k = 0; k < (int)ez; ++k)
    for (int j = 0; j < (int)ey; ++j)
      for (int i = 0; i < (int)ex; ++i) {
        int need;
        int kd = point_delay(p, d, i, j, k, kf, &need);
        if (!need) continue;
        double dd[5];
        or_buffer_dudt(p->order, m - 1, (double)kd, dd);
        int gx = wrapi(d->ox + i - d->g, p->nx), gy = wrapi(d->oy + j - d->g, p->ny);
        int gz = wrapi(d->oz + k - d->gz, p->nz);
        size_t gq = (size_t)gx + (size_t)p->nx * (gy + (size_t)p->ny * gz);
        size_t q = (size_t)i + ex * (j + ey * k);
        for (int v = 0; v < NV; ++v) {
          double s = 0.0; /* = dt * dU/dt|_buf^(m-1) */
          for (int l = 0; l < C; ++l) s += dd[l] * H(h, n - kd - l)[v * N + gq];
          double qn = A[m - 1] * hb->qb[v * ne + q] + s;
          hb->qb[v * ne + q] = qn;
          hb->ub[v * ne + q] += B[m - 1] * qn;
        }
      }
}

/* One filter pass along axis `ax` over all sub-domains: Uin -> Uout. */
static void filter_pass(const or_params* p, int ax, const double* Uin, double* Uout, int mode,
                        const hist_t* h, long n, int** kfs, int nsub) {
  const size_t N = (size_t)p->nx * p->ny * p->nz;
  const int C = or_levels(p->order);
  const int nn[3] = {p->nx, p->ny, p->nz};
  memcpy(Uout, Uin, sizeof(double) * NV * N);
#pragma omp parallel for schedule(dynamic)
  for (int s = 0; s < nsub; ++s) {
    subdom d;
    make_subdom(p, s, 0, &d);
    const int o[3] = {d.ox, d.oy, d.oz}, sz[3] = {d.sx, d.sy, d.sz};
    const int* kf = kfs[s];
    int len = sz[ax];
    double* line = (double*)malloc(sizeof(double) * (len + 10));
    double* out = (double*)malloc(sizeof(double) * len);
    int a1 = (ax + 1) % 3, a2 = (ax + 2) % 3;
    for (int t2 = 0; t2 < sz[a2]; ++t2)
      for (int t1 = 0; t1 < sz[a1]; ++t1)
        for (int v = 0; v < NV; ++v) {
          for (int t = -5; t < len + 5; ++t) {
            int c[3];
            c[ax] = wrapi(o[ax] + t, nn[ax]);
            c[a1] = o[a1] + t1;
            c[a2] = o[a2] + t2;
            size_t gq = (size_t)c[0] + (size_t)p->nx * (c[1] + (size_t)p->ny * c[2]);
            double val;
            if (t >= 0 && t < len) val = Uin[v * N + gq];
            else {
              int f = 2 * ax + (t < 0 ? 0 : 1);
              int kd = kf[f];
              if (mode == 0) val = Uin[v * N + gq];
              else if (mode == 2) val = H(h, n - kd)[v * N + gq];
              else {
                /* extrapolate the visible levels to t_{n+1}: delay k+1 relative to n+1 */
                double cw[5];
                or_extrap_weights(p->order, (double)(kd + 1), cw);
                double sacc = 0.0;
                for (int l = 0; l < C; ++l) sacc += cw[l] * H(h, n - kd - l)[v * N + gq];
                val = sacc;
              }
            }
            line[t + 5] = val;
          }
          or_filter_line(len, p->alpha_f, line, out);
          for (int t = 0; t < len; ++t) {
            int c[3];
            c[ax] = o[ax] + t;
            c[a1] = o[a1] + t1;
            c[a2] = o[a2] + t2;
            size_t gq = (size_t)c[0] + (size_t)p->nx * (c[1] + (size_t)p->ny * c[2]);
            Uout[v * N + gq] = out[t];
          }
        }
    free(line);
    free(out);
  }
}

/* Ring depth needed for a run: largest delay + C + 1. */
static int ring_depth(const or_params* p) {
  int C = or_levels(p->order);
  int kmax = 0;
  if (p->algo == 1) kmax = p->caa_L - 1;
  if (p->algo == 2) kmax = p->kmax;
  return kmax + C + 1;
}

/* Initial-history state for a resumed run: levels n0 - R + 1 .. n0 may be passed in `hist_in`
 * ([R][5][N], level n0 - R + 1 first); NULL means a fresh start at n0 = 0 from U0. */

/*
 * Advance `nsteps` steps starting from step index n0 with state U (in/out).
 * delays: SAA table int8 [n0 + nsteps][nsub][6] (ignored for SA/CAA).
 * diag (optional): per step [nsteps][8] = KE, enstrophy, sum rho, sum rho u, sum rho v,
 *                  sum rho w, sum rho E, nan-flag (after the step).
 * Returns 0 on success, nonzero on invalid input.
 */
int or_diagnostics(const or_params* p, const double* U, double* out);

int or_run(const or_params* p, double* U, const int8_t* delays, long n0, long nsteps, const double* hist_in,
           double* diag) {
  const size_t N = (size_t)p->nx * p->ny * p->nz;
  const int nsub = p->px * p->py * p->pz;
  const int C = or_levels(p->order);
  const int r = (p->order == 4) ? 2 : 1;
  const int g = p->viscous ? 2 * r : r;
  double A[5], B[5];
  const int S = or_lserk(p->order, A, B);
  /* validation */
  for (int s = 0; s < nsub; ++s) {
    subdom d;
    make_subdom(p, s, g, &d);
    int need = g > (p->filter ? 5 : 0) ? g : (p->filter ? 5 : 0);
    if (d.sx < need || d.sy < need || (p->nz > 1 && d.sz < need)) return 1;
  }
  if (p->algo == 1 && p->caa_L < 1) return 2;
  hist_t h;
  h.R = ring_depth(p);
  h.lev = (double**)malloc(sizeof(double*) * h.R);
  for (int i = 0; i < h.R; ++i) h.lev[i] = (double*)calloc(NV * N, sizeof(double));
  if (hist_in) {
    for (int i = 0; i < h.R; ++i) {
      long lvl = n0 - h.R + 1 + i;
      if (lvl >= 0) memcpy(h.lev[lvl % h.R], hist_in + (size_t)i * NV * N, sizeof(double) * NV * N);
    }
  }
  memcpy(h.lev[n0 % h.R], U, sizeof(double) * NV * N);

  double* Ucur = (double*)malloc(sizeof(double) * NV * N);
  double* Unew = (double*)malloc(sizeof(double) * NV * N);
  double* Q = (double*)malloc(sizeof(double) * NV * N);
  double* Mg = metric_field(p);
  int** kfs = (int**)malloc(sizeof(int*) * nsub);
  for (int s = 0; s < nsub; ++s) kfs[s] = (int*)malloc(sizeof(int) * 6);
  halo_t* hbs = (halo_t*)calloc(nsub, sizeof(halo_t));

  for (long n = n0; n < n0 + nsteps; ++n) {
    int mode = (p->algo == 0 || n < C) ? 0 : (p->at ? 1 : 2);
    for (int s = 0; s < nsub; ++s)
      for (int f = 0; f < 6; ++f) {
        int k = (mode == 0) ? 0 : raw_delay(p, delays, nsub, n, s, f);
        long cap = n - C + 1;
        if (k > cap) k = (int)cap;
        if (k < 0) k = 0;
        kfs[s][f] = k;
      }
    memcpy(Ucur, H(&h, n), sizeof(double) * NV * N);
    memset(Q, 0, sizeof(double) * NV * N);
    for (int m = 1; m <= S; ++m) {
#pragma omp parallel
      {
        work_t w;
        memset(&w, 0, sizeof(w));
#pragma omp for schedule(dynamic)
        for (int s = 0; s < nsub; ++s) {
          subdom d;
          make_subdom(p, s, g, &d);
          size_t ne = (size_t)d.ex * d.ey * d.ez;
          work_reserve(&w, ne);
          if (mode == 1) {
            if (hbs[s].cap < ne) {
              free(hbs[s].ub); free(hbs[s].qb);
              hbs[s].ub = (double*)malloc(sizeof(double) * NV * ne);
              hbs[s].qb = (double*)malloc(sizeof(double) * NV * ne);
              hbs[s].cap = ne;
            }
            if (m == 1) {
              halo_init(p, &d, &h, n, kfs[s], &hbs[s]);
              if (p->mlp) halo_init_learned(p, &d, s, &h, n, kfs[s], &hbs[s]);
            }
          }
          fill_ext(p, &d, Ucur, mode, &h, n, kfs[s], &hbs[s], &w);
          size_t no = (size_t)d.sx * d.sy * d.sz;
          double* R = (double*)malloc(sizeof(double) * NV * no);
          if (Mg) rhs_ext_curv(p, &d, Mg, &w, R);
          else rhs_ext(p, &d, &w, R);
          /* Eq. 3: Q^(m) = A_m Q^(m-1) + dt R(U^(m-1));  U^(m) = U^(m-1) + B_m Q^(m) */
          for (int v = 0; v < NV; ++v)
            for (int k = 0; k < d.sz; ++k)
              for (int j = 0; j < d.sy; ++j)
                for (int i = 0; i < d.sx; ++i) {
                  size_t gq = (size_t)(d.ox + i) + (size_t)p->nx * ((d.oy + j) + (size_t)p->ny * (d.oz + k));
                  size_t o = (size_t)i + (size_t)d.sx * (j + (size_t)d.sy * k);
                  double qn = A[m - 1] * Q[v * N + gq] + p->dt * R[v * no + o];
                  Q[v * N + gq] = qn;
                  Unew[v * N + gq] = Ucur[v * N + gq] + B[m - 1] * qn;
                }
          free(R);
          if (mode == 1 && m <= S - 1) halo_update(p, &d, &h, n, kfs[s], m, A, B, &hbs[s]);
        }
        work_free(&w);
      }
      double* t = Ucur; Ucur = Unew; Unew = t;
    }
    if (p->filter) {
      int nd = p->nz > 1 ? 3 : 2;
      for (int ax = 0; ax < nd; ++ax) {
        filter_pass(p, ax, Ucur, Unew, mode, &h, n, kfs, nsub);
        double* t = Ucur; Ucur = Unew; Unew = t;
      }
    }
    memcpy(h.lev[(n + 1) % h.R], Ucur, sizeof(double) * NV * N);
    if (diag) or_diagnostics(p, Ucur, diag + (size_t)(n - n0) * 8);
  }
  memcpy(U, Ucur, sizeof(double) * NV * N);
  for (int i = 0; i < h.R; ++i) free(h.lev[i]);
  free(h.lev);
  free(Ucur); free(Unew); free(Q); free(Mg);
  for (int s = 0; s < nsub; ++s) { free(kfs[s]); free(hbs[s].ub); free(hbs[s].qb); }
  free(kfs); free(hbs);
  return 0;
}

/* R(U) of the whole periodic field in synchronous mode (halos = current neighbour values). */
int or_rhs(const or_params* p, const double* U, double* Rout) {
  const size_t N = (size_t)p->nx * p->ny * p->nz;
  const int nsub = p->px * p->py * p->pz;
  const int r = (p->order == 4) ? 2 : 1;
  const int g = p->viscous ? 2 * r : r;
  int kf[6] = {0, 0, 0, 0, 0, 0};
  for (int s = 0; s < nsub; ++s) {
    subdom d;
    make_subdom(p, s, g, &d);
    if (d.sx < g || d.sy < g || (p->nz > 1 && d.sz < g)) return 1;
  }
  double* Mg = metric_field(p);
#pragma omp parallel
  {
    work_t w;
    memset(&w, 0, sizeof(w));
#pragma omp for schedule(dynamic)
    for (int s = 0; s < nsub; ++s) {
      subdom d;
      make_subdom(p, s, g, &d);
      work_reserve(&w, (size_t)d.ex * d.ey * d.ez);
      fill_ext(p, &d, U, 0, NULL, 0, kf, NULL, &w);
      size_t no = (size_t)d.sx * d.sy * d.sz;
      double* R = (double*)malloc(sizeof(double) * NV * no);
      if (Mg) rhs_ext_curv(p, &d, Mg, &w, R);
      else rhs_ext(p, &d, &w, R);
      for (int v = 0; v < NV; ++v)
        for (int k = 0; k < d.sz; ++k)
          for (int j = 0; j < d.sy; ++j)
            for (int i = 0; i < d.sx; ++i) {
              size_t gq = (size_t)(d.ox + i) + (size_t)p->nx * ((d.oy + j) + (size_t)p->ny * (d.oz + k));
              Rout[v * N + gq] = R[v * no + (size_t)i + (size_t)d.sx * (j + (size_t)d.sy * k)];
            }
      free(R);
    }
    work_free(&w);
  }
  free(Mg);
  return 0;
}

/* Volume-averaged kinetic energy and enstrophy (Sec. 5.2, rho_0 = 1) with vorticity from the CD
 * scheme on the periodic field, cell-volume-weighted totals of the conserved variables, and a
 * non-finite flag.  out[8] = {K, eps, sum rho, sum rho u, sum rho v, sum rho w, sum rho E, nan}.
 * On a curvilinear grid the cell volume is J^-1 and the averages are volume-weighted; velocity
 * derivatives are taken in index space and mapped by the metric terms. */
int or_diagnostics(const or_params* p, const double* U, double* out) {
  const int nx = p->nx, ny = p->ny, nz = p->nz;
  const size_t N = (size_t)nx * ny * nz;
  double* Mg = metric_field(p);
  const double dV0 = p->dx * p->dy * (nz > 1 ? p->dz : 1.0);
  double ke = 0, ens = 0, vol = 0, tot[5] = {0, 0, 0, 0, 0};
  int bad = 0;
  const int order = p->order;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t q = (size_t)i + (size_t)nx * (j + (size_t)ny * k);
        const double dV = Mg ? Mg[5 * N + q] : dV0;
        double rho = U[q];
        double u = U[N + q] / rho, v = U[2 * N + q] / rho, w = U[3 * N + q] / rho;
        for (int c = 0; c < 5; ++c) {
          if (!isfinite(U[c * N + q])) bad = 1;
          tot[c] += U[c * N + q] * dV;
        }
        const double wv = Mg ? dV : 1.0; /* Cartesian: plain point average */
        vol += wv;
        ke += 0.5 * rho * (u * u + v * v + w * w) * wv;
        /* velocity derivative along axis a of component c at (i,j,k), periodic CD */
        double dvel[3][3];
        for (int c = 0; c < 3; ++c)
          for (int a = 0; a < 3; ++a) {
            int n_a = a == 0 ? nx : (a == 1 ? ny : nz);
            if (n_a == 1) { dvel[c][a] = 0.0; continue; }
            double hh = Mg ? 1.0 : (a == 0 ? p->dx : (a == 1 ? p->dy : p->dz));
            double f[5];
            for (int o = -2; o <= 2; ++o) {
              int ii = i, jj = j, kk = k;
              if (a == 0) ii = wrapi(i + o, nx);
              if (a == 1) jj = wrapi(j + o, ny);
              if (a == 2) kk = wrapi(k + o, nz);
              size_t qq = (size_t)ii + (size_t)nx * (jj + (size_t)ny * kk);
              f[o + 2] = U[(1 + c) * N + qq] / U[qq];
            }
            if (order == 4)
              dvel[c][a] = ((-1.0 / 3.0) * (f[4] - f[0]) / 4.0 + (4.0 / 3.0) * (f[3] - f[1]) / 2.0) / hh;
            else
              dvel[c][a] = (f[3] - f[1]) / (2.0 * hh);
          }
        if (Mg) {
          /* d u_c / d x_j = J sum_a (metric row a)_j d u_c / d xi_a */
          const double J = 1.0 / Mg[5 * N + q];
          const double m[3][3] = {{Mg[q], Mg[N + q], 0.0}, {Mg[2 * N + q], Mg[3 * N + q], 0.0}, {0.0, 0.0, Mg[4 * N + q]}};
          double dphys[3][3];
          for (int c = 0; c < 3; ++c)
            for (int jj = 0; jj < 3; ++jj)
              dphys[c][jj] = J * (m[0][jj] * dvel[c][0] + m[1][jj] * dvel[c][1] + m[2][jj] * dvel[c][2]);
          memcpy(dvel, dphys, sizeof(dvel));
        }
        double wx = dvel[2][1] - dvel[1][2], wy = dvel[0][2] - dvel[2][0], wz = dvel[1][0] - dvel[0][1];
        ens += 0.5 * rho * (wx * wx + wy * wy + wz * wz) * wv;
      }
  out[0] = ke / vol;
  out[1] = ens / vol;
  for (int c = 0; c < 5; ++c) out[2 + c] = tot[c];
  out[7] = bad ? 1.0 : 0.0;
  free(Mg);
  return 0;
}

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void or_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
