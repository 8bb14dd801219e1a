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
 *   - Eq. 2 / App. B: explicit central differences CD2 (a=1,b=0) and CD4 (a=4/3,b=-1/3); the
 *     sixth-order compact scheme (alpha=1/3, a=14/9, b=1/9) for the Euler fluxes, per sub-domain
 *     line with an explicit sixth-order closure at the first halo point (a reading).
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
 *   - Multi-block grids: blocks joined at node-disjoint interfaces (tangential index aligned or
 *     reversed, spanwise counts equal or different: four-point Lagrange interpolation in z),
 *     ending at no-slip adiabatic walls (mirrored state, momentum negated; wall points keep zero
 *     momentum through the stages and the filter), far fields (a given state) or outflows (the
 *     face values repeated).  Halo values beyond a block face resolve axis by axis, x then y then
 *     z; metric terms beyond a non-periodic face come from the grid continued across it
 *     (interfaces) or reflected through the boundary point (physical faces).  A halo source is
 *     the PE's own value (current) when reached by a wall mirror or an outflow copy within the
 *     sub-domain; otherwise it is a neighbour's, seen with the face's delay.
 *
 * Layout: a state array holds every block's U[5][nz][ny][nx] (structure of arrays, FP64) one
 * after the other; a single-grid run is one block, periodic in all directions.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NV 5

/* Face of a block (faces 0..5 = -x, +x, -y, +y, -z, +z).  Types: periodic (the block wraps onto
 * itself), interface (to face nf of block nb; node-disjoint: the first point beyond the face is
 * the neighbour's first point inside its face; rev = 1 when the tangential in-plane index runs
 * the other way on the neighbour; the neighbour's coordinates continue the block's grid after
 * adding shift, nonzero where the interface closes a periodic direction), no-slip adiabatic wall (the points on the face are wall
 * points; beyond it the state is mirrored about the face with the momentum negated), far field
 * (the given conserved state beyond the face) and outflow (the face values repeated beyond it). */
enum { OR_PERIODIC = 0, OR_INTERFACE = 1, OR_WALL = 2, OR_FARFIELD = 3, OR_OUTFLOW = 4 };
typedef struct {
  int type;
  int nb, nf, rev;
  double state[5];
  double shift[2]; /* interface: coordinate jump (x, y) added to the neighbour's points */
} or_face;

/* One block of a multi-block run: its grid, its split into sub-domains and its six faces
 * (z faces periodic: blocks are extruded along z). */
typedef struct {
  int nx, ny, nz, px, py, pz;
  double dx, dy, dz;
  const double* grid_xy;  /* [2][ny][nx] point coordinates, or NULL (uniform Cartesian) */
  double grid_shift[4];   /* coordinate jumps across periodic wraps in xi (x, y) and eta (x, y) */
  or_face face[6];
} or_block;

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
  /* multi-block run: nblocks > 0 blocks replace the single periodic grid above (whose grid,
   * split and spacing fields are then ignored); states are stored block after block */
  int nblocks;
  const or_block* blocks;
  /* 1: the flux divergence by the sixth-order compact scheme of Eq. 2 (alpha = 1/3) with an
   * explicit sixth-order closure at the first halo point of every sub-domain line (Euler,
   * single periodic Cartesian grid, LSERK4 / AT4 in time: order = 4); halo depth 4 */
  int compact;
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

/* Halo depth of the sub-domains: 2r for the viscous CD operator, r for the Euler one, 4 for the
 * compact scheme (its sixth-order closure at the first halo point reads three points beyond). */
static int halo_g(const or_params* p) {
  const int r = (p->order == 4) ? 2 : 1;
  if (p->compact) return 4;
  return p->viscous ? 2 * r : r;
}

/* Sixth-order compact first derivative (Eq. 2 with alpha = 1/3, a = 14/9, b = 1/9) on one
 * sub-domain line of n points spaced h, from f[0 .. n+7] (point i at f[i + 4]: four halo values on
 * each side).  The tridiagonal system for the n owned derivatives is closed by the explicit
 * sixth-order central difference (45, -9, 1)/60h at the first halo point on each side (the paper
 * prints no closure for its compact schemes at PE boundaries; halo values are the AT ones on
 * asynchronous steps).  Solved by the Thomas algorithm.  d[0 .. n-1] receives the derivatives. */
void or_compact_line(int n, double h, const double* f, double* d) {
  if (n < 1) return;
  const double al = 1.0 / 3.0, a = 14.0 / 9.0, b = 1.0 / 9.0;
  const double* F = f + 4;
  const double dl = (45.0 * (F[0] - F[-2]) - 9.0 * (F[1] - F[-3]) + (F[2] - F[-4])) / (60.0 * h);
  const double dr = (45.0 * (F[n + 1] - F[n - 1]) - 9.0 * (F[n + 2] - F[n - 2]) + (F[n + 3] - F[n - 3])) / (60.0 * h);
  double* cp = (double*)malloc(sizeof(double) * (size_t)n);
  double* rh = (double*)malloc(sizeof(double) * (size_t)n);
  for (int i = 0; i < n; ++i) rh[i] = a * (F[i + 1] - F[i - 1]) / (2.0 * h) + b * (F[i + 2] - F[i - 2]) / (4.0 * h);
  rh[0] -= al * dl;
  rh[n - 1] -= al * dr;
  /* forward elimination (unit diagonal, off-diagonals alpha), then back substitution */
  cp[0] = al;
  for (int i = 1; i < n; ++i) {
    const double m = 1.0 - al * cp[i - 1];
    cp[i] = al / m;
    rh[i] = (rh[i] - al * rh[i - 1]) / m;
  }
  d[n - 1] = rh[n - 1];
  for (int i = n - 2; i >= 0; --i) d[i] = rh[i] - cp[i] * d[i + 1];
  free(cp);
  free(rh);
}

typedef struct {
  int ox, oy, oz, sx, sy, sz;  /* owned box */
  int g, gz;                   /* ghost depth in x/y and in z (0 in 2-D) */
  int ex, ey, ez;              /* extended dims */
  int b;                       /* block of the sub-domain */
  int phys[6];                 /* 1: the face lies on a physical boundary of the block */
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
  d->b = 0;
  for (int f = 0; f < 6; ++f) d->phys[f] = 0;
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
/* ---------------------------------------------------------------- blocks, faces, halo sources
 * The run's blocks (a single-grid run is one block with six periodic faces), each block's state
 * stored after the previous one's ([5][nz][ny][nx] per block), sub-domains numbered block after
 * block.  Values beyond a block face follow the face's type (see or_face); an interface that
 * joins blocks of different spanwise counts gives the receiving point the neighbour's values at
 * the same spanwise position, by four-point Lagrange interpolation between the neighbour's
 * points (a point that falls on a neighbour point takes it alone). */
typedef struct {
  int nb, nsub;
  or_block* b;    /* the blocks */
  or_params* pb;  /* per block: a copy of the run's parameters with the block's grid and split */
  size_t* base;   /* offset of each block's state in a state array (doubles) */
  size_t* np;     /* points of each block */
  int* sid0;      /* first sub-domain of each block (nb + 1 entries) */
  size_t Ntot;    /* points of all blocks */
  int g;          /* halo depth of the stage (2r viscous, r Euler) */
  double** M;     /* per block: metric terms on the plane extended by g, or NULL (Cartesian) */
} topo_t;

static inline size_t at_pt(const topo_t* T, int b, int v, int i, int j, int k) {
  const or_block* B = &T->b[b];
  return T->base[b] + (size_t)v * T->np[b] + (size_t)i + (size_t)B->nx * ((size_t)j + (size_t)B->ny * (size_t)k);
}

static int block_of(const topo_t* T, int s, int* local) {
  int b = 0;
  while (b + 1 < T->nb && s >= T->sid0[b + 1]) ++b;
  *local = s - T->sid0[b];
  return b;
}

/* Sub-domain s with its block and the physical boundaries among its faces. */
static void make_sub(const topo_t* T, int s, int g, subdom* d) {
  int local;
  const int b = block_of(T, s, &local);
  make_subdom(&T->pb[b], local, g, d);
  d->b = b;
  const or_block* B = &T->b[b];
  const int lo[3] = {d->ox, d->oy, d->oz}, hi[3] = {d->ox + d->sx, d->oy + d->sy, d->oz + d->sz};
  const int n[3] = {B->nx, B->ny, B->nz};
  for (int a = 0; a < 3; ++a) {
    d->phys[2 * a] = lo[a] == 0 && B->face[2 * a].type >= OR_WALL;
    d->phys[2 * a + 1] = hi[a] == n[a] && B->face[2 * a + 1].type >= OR_WALL;
  }
}

/* sign of conserved variable v after a wall reflection */
static inline double refl_sign(int v, int flip) { return (flip && v >= 1 && v <= 3) ? -1.0 : 1.0; }

#define OR_MAXT 4
typedef struct {
  int b, i, j, k;
  int flip;     /* momentum negated (odd number of wall reflections) */
  int crossed;  /* the path crossed a periodic wrap or a block interface */
  double w;
} or_term;

/* Four-point Lagrange weights at fraction th of the way from node 0 to node 1 (nodes -1..2). */
static void lagrange4(double th, double* l) {
  l[0] = -th * (th - 1.0) * (th - 2.0) / 6.0;
  l[1] = (th + 1.0) * (th - 1.0) * (th - 2.0) / 2.0;
  l[2] = -(th + 1.0) * th * (th - 2.0) / 2.0;
  l[3] = (th + 1.0) * th * (th - 1.0) / 6.0;
}

/* Sources of the state at point (i, j, k) of block b's index space (any point within a halo
 * depth of the block): U_v = sum_t w_t s_v(flip_t) U_v(term t) + cst_v.  The axes are resolved
 * in the order x, y, z, each in the frame of the block reached so far.  Returns the number of
 * terms, or -1 when more than OR_MAXT would be needed or the point does not resolve. */
static int resolve_state(const topo_t* T, int b, int i, int j, int k, or_term* t, double* cst) {
  int n = 1;
  t[0].b = b; t[0].i = i; t[0].j = j; t[0].k = k; t[0].flip = 0; t[0].crossed = 0; t[0].w = 1.0;
  for (int v = 0; v < NV; ++v) cst[v] = 0.0;
  for (int q = 0; q < n; ++q) {
    int hop;
    for (hop = 0; hop < 16; ++hop) {
      or_term* x = &t[q];
      const or_block* B = &T->b[x->b];
      int c[3] = {x->i, x->j, x->k};
      const int nn[3] = {B->nx, B->ny, B->nz};
      int a = -1;
      for (int e = 0; e < 3; ++e)
        if (c[e] < 0 || c[e] >= nn[e]) { a = e; break; }
      if (a < 0) break;
      const int side = c[a] < 0 ? 0 : 1;
      const or_face* F = &B->face[2 * a + side];
      if (F->type == OR_PERIODIC) {
        c[a] = wrapi(c[a], nn[a]);
        x->crossed = 1;
      } else if (F->type == OR_WALL) {
        c[a] = side == 0 ? -c[a] : 2 * (nn[a] - 1) - c[a];
        x->flip ^= 1;
      } else if (F->type == OR_OUTFLOW) {
        c[a] = side == 0 ? 0 : nn[a] - 1;
      } else if (F->type == OR_FARFIELD) {
        for (int v = 0; v < NV; ++v) cst[v] += x->w * refl_sign(v, x->flip) * F->state[v];
        t[q] = t[n - 1];
        --n;
        --q;
        break;
      } else if (F->type == OR_INTERFACE && a < 2) {
        const or_block* B2 = &T->b[F->nb];
        const int m = side == 0 ? -c[a] : c[a] - (nn[a] - 1);  /* depth beyond the face */
        const int a2 = F->nf / 2, s2 = F->nf % 2, ta = 1 - a, ta2 = 1 - a2;
        const int n2[3] = {B2->nx, B2->ny, B2->nz};
        int c2[3];
        c2[a2] = s2 == 0 ? m - 1 : n2[a2] - m;
        c2[ta2] = F->rev ? nn[ta] - 1 - c[ta] : c[ta];
        c2[2] = c[2];
        x->b = F->nb;
        x->crossed = 1;
        if (n2[2] != nn[2]) {
          /* spanwise position c[2] nz2 / nz on the neighbour */
          const long num = (long)c[2] * n2[2];
          long z0 = num / nn[2];
          if (z0 * nn[2] > num) --z0;
          const long rem = num - z0 * nn[2];
          c2[2] = (int)z0;
          if (rem != 0) {
            if (n + 3 > OR_MAXT) return -1;
            double l[4];
            lagrange4((double)rem / (double)nn[2], l);
            const or_term base = *x;
            for (int o = 0; o < 4; ++o) {
              or_term* y = (o == 0) ? x : &t[n + o - 1];
              *y = base;
              y->i = c2[0]; y->j = c2[1]; y->k = (int)z0 + o - 1;
              y->w = base.w * l[o];
            }
            n += 3;
            continue;
          }
        }
        c[0] = c2[0]; c[1] = c2[1]; c[2] = c2[2];
      } else {
        return -1;
      }
      x->i = c[0]; x->j = c[1]; x->k = c[2];
    }
    if (hop == 16) return -1;
  }
  return n;
}

/* Point coordinates (x, y) at (i, j) of curvilinear block b's plane, for points up to a few halo
 * depths outside it: a periodic face wraps the index and adds the coordinate jump, an interface
 * continues into the neighbour (which must be curvilinear too), a physical face reflects the grid
 * through the boundary point, x(-m) = 2 x(0) - x(m).  Returns nonzero if it does not resolve. */
static int coord_ext(const topo_t* T, int b, int i, int j, int depth, double* xy) {
  if (depth > 8) return 1;
  const or_block* B = &T->b[b];
  const int nn[2] = {B->nx, B->ny};
  int wi = 0, wj = 0;
  for (int hop = 0; hop < 4; ++hop) {
    int c[2] = {i, j};
    int a = -1;
    for (int e = 0; e < 2; ++e)
      if (c[e] < 0 || c[e] >= nn[e]) { a = e; break; }
    if (a < 0) break;
    const int side = c[a] < 0 ? 0 : 1;
    const or_face* F = &B->face[2 * a + side];
    double r0[2], r1[2];
    if (F->type == OR_PERIODIC) {
      const int w = wrapi(c[a], nn[a]);
      if (a == 0) wi += (c[a] - w) / nn[a];
      else wj += (c[a] - w) / nn[a];
      c[a] = w;
      i = c[0]; j = c[1];
      continue;
    }
    if (F->type == OR_INTERFACE) {
      const or_block* B2 = &T->b[F->nb];
      const int m = side == 0 ? -c[a] : c[a] - (nn[a] - 1);
      const int a2 = F->nf / 2, s2 = F->nf % 2, ta = 1 - a, ta2 = 1 - a2;
      const int n2[2] = {B2->nx, B2->ny};
      int c2[2];
      c2[a2] = s2 == 0 ? m - 1 : n2[a2] - m;
      c2[ta2] = F->rev ? nn[ta] - 1 - c[ta] : c[ta];
      if (coord_ext(T, F->nb, c2[0], c2[1], depth + 1, r0)) return 1;
      for (int q = 0; q < 2; ++q) xy[q] = r0[q] + F->shift[q] + wi * B->grid_shift[q] + wj * B->grid_shift[2 + q];
      return 0;
    }
    /* physical boundary: reflection through the boundary point */
    int cb[2] = {c[0], c[1]}, cm[2] = {c[0], c[1]};
    cb[a] = side == 0 ? 0 : nn[a] - 1;
    cm[a] = side == 0 ? -c[a] : 2 * (nn[a] - 1) - c[a];
    if (coord_ext(T, b, cb[0], cb[1], depth + 1, r0) || coord_ext(T, b, cm[0], cm[1], depth + 1, r1)) return 1;
    for (int q = 0; q < 2; ++q) xy[q] = 2.0 * r0[q] - r1[q] + wi * B->grid_shift[q] + wj * B->grid_shift[2 + q];
    return 0;
  }
  if (i < 0 || i >= nn[0] || j < 0 || j >= nn[1]) return 1;
  for (int q = 0; q < 2; ++q)
    xy[q] = B->grid_xy[(size_t)q * nn[0] * nn[1] + (size_t)i + (size_t)nn[0] * j] + wi * B->grid_shift[q] +
            wj * B->grid_shift[2 + q];
  return 0;
}

#define NM 6 /* xi^_x, xi^_y, eta^_x, eta^_y, zeta^_z, J^-1 */

/* Metric terms at point (i, j) of block b's plane (in the block's own index frame); the
 * coordinate derivatives by the scheme of Eq. 2 in index space.  Nonzero if a coordinate does
 * not resolve. */
static int metric_point(const topo_t* T, int b, int i, int j, double* m) {
  const or_params* p = &T->pb[b];
  double d[2][2]; /* d[c][axis] = d (x, y)_c / d xi_axis */
  for (int axis = 0; axis < 2; ++axis) {
    double f[5][2];
    for (int o = -2; o <= 2; ++o) {
      if (p->order != 4 && (o == -2 || o == 2)) { f[o + 2][0] = f[o + 2][1] = 0.0; continue; }
      if (coord_ext(T, b, axis == 0 ? i + o : i, axis == 0 ? j : j + o, 0, f[o + 2])) return 1;
    }
    for (int c = 0; c < 2; ++c) {
      if (p->order == 4)
        d[c][axis] = (-1.0 / 3.0) * (f[4][c] - f[0][c]) / 4.0 + (4.0 / 3.0) * (f[3][c] - f[1][c]) / 2.0;
      else
        d[c][axis] = (f[3][c] - f[1][c]) / 2.0;
    }
  }
  const double x_xi = d[0][0], x_eta = d[0][1], y_xi = d[1][0], y_eta = d[1][1];
  const double zz = p->nz > 1 ? p->dz : 1.0;
  const double det = x_xi * y_eta - x_eta * y_xi;
  m[0] = y_eta * zz; m[1] = -x_eta * zz; m[2] = -y_xi * zz; m[3] = x_xi * zz; m[4] = det; m[5] = zz * det;
  return 0;
}

/* Metric terms of curvilinear block b on its plane extended by g points on every side,
 * [NM][(nx + 2g)(ny + 2g)]: a point beyond a periodic face takes the wrapped point's values;
 * beyond another face, the values of the grid continued as coord_ext continues it, to the
 * stencil radius (deeper points, which no flux reads, are NaN). */
static double* metric_plane(const topo_t* T, int b) {
  const or_block* B = &T->b[b];
  if (!B->grid_xy) return NULL;
  const int g = T->g, r = T->pb[b].order == 4 ? 2 : 1;
  const int ex = B->nx + 2 * g, ey = B->ny + 2 * g;
  const size_t pl = (size_t)ex * ey;
  double* M = (double*)malloc(sizeof(double) * NM * pl);
  for (int jj = -g; jj < B->ny + g; ++jj)
    for (int ii = -g; ii < B->nx + g; ++ii) {
      int i = ii, j = jj;
      if ((i < 0 && B->face[0].type == OR_PERIODIC) || (i >= B->nx && B->face[1].type == OR_PERIODIC)) i = wrapi(i, B->nx);
      if ((j < 0 && B->face[2].type == OR_PERIODIC) || (j >= B->ny && B->face[3].type == OR_PERIODIC)) j = wrapi(j, B->ny);
      const int di = i < 0 ? -i : (i >= B->nx ? i - B->nx + 1 : 0);
      const int dj = j < 0 ? -j : (j >= B->ny ? j - B->ny + 1 : 0);
      double m[NM];
      if (di > r || dj > r || metric_point(T, b, i, j, m))
        for (int c = 0; c < NM; ++c) m[c] = NAN;
      const size_t q = (size_t)(ii + g) + (size_t)ex * (jj + g);
      for (int c = 0; c < NM; ++c) M[c * pl + q] = m[c];
    }
  return M;
}

static inline double metric_at(const topo_t* T, int b, int c, int i, int j) {
  const or_block* B = &T->b[b];
  const int g = T->g, ex = B->nx + 2 * g;
  const size_t pl = (size_t)ex * (B->ny + 2 * g);
  return T->M[b][(size_t)c * pl + (size_t)(i + g) + (size_t)ex * (j + g)];
}

static void topo_free(topo_t* T) {
  if (T->M)
    for (int b = 0; b < T->nb; ++b) free(T->M[b]);
  free(T->M); free(T->b); free(T->pb); free(T->base); free(T->np); free(T->sid0);
  memset(T, 0, sizeof(*T));
}

/* The run's blocks: validated faces (z periodic; interfaces paired both ways, in-plane, with
 * equal tangential counts; curvilinear only to curvilinear; between Cartesian blocks only
 * opposite faces of one axis with the tangential index unreversed), metric planes, and every
 * halo point within depth gmax of a block resolvable.  Nonzero on an invalid description. */
static int topo_build(const or_params* p, int g, int gmax, topo_t* T) {
  memset(T, 0, sizeof(*T));
  const int nb = p->nblocks > 0 ? p->nblocks : 1;
  T->nb = nb;
  T->g = g;
  T->b = (or_block*)calloc(nb, sizeof(or_block));
  T->pb = (or_params*)calloc(nb, sizeof(or_params));
  T->base = (size_t*)calloc(nb, sizeof(size_t));
  T->np = (size_t*)calloc(nb, sizeof(size_t));
  T->sid0 = (int*)calloc(nb + 1, sizeof(int));
  T->M = (double**)calloc(nb, sizeof(double*));
  if (p->nblocks > 0) {
    memcpy(T->b, p->blocks, sizeof(or_block) * nb);
  } else {
    or_block* B = &T->b[0];
    B->nx = p->nx; B->ny = p->ny; B->nz = p->nz; B->px = p->px; B->py = p->py; B->pz = p->pz;
    B->dx = p->dx; B->dy = p->dy; B->dz = p->dz;
    B->grid_xy = p->grid_xy;
    for (int q = 0; q < 4; ++q) B->grid_shift[q] = p->grid_shift[q];
    for (int f = 0; f < 6; ++f) B->face[f].type = OR_PERIODIC;
  }
  size_t off = 0;
  int s0 = 0;
  for (int b = 0; b < nb; ++b) {
    const or_block* B = &T->b[b];
    if (B->nx < 1 || B->ny < 1 || B->nz < 1 || B->px < 1 || B->py < 1 || B->pz < 1) return 10;
    or_params* q = &T->pb[b];
    *q = *p;
    q->nx = B->nx; q->ny = B->ny; q->nz = B->nz; q->px = B->px; q->py = B->py; q->pz = B->pz;
    q->dx = B->dx; q->dy = B->dy; q->dz = B->dz;
    q->grid_xy = B->grid_xy;
    for (int k = 0; k < 4; ++k) q->grid_shift[k] = B->grid_shift[k];
    q->nblocks = 0;
    q->blocks = NULL;
    T->base[b] = off;
    T->np[b] = (size_t)B->nx * B->ny * B->nz;
    off += NV * T->np[b];
    T->Ntot += T->np[b];
    T->sid0[b] = s0;
    s0 += B->px * B->py * B->pz;
  }
  T->sid0[nb] = s0;
  T->nsub = s0;
  for (int b = 0; b < nb; ++b) {
    const or_block* B = &T->b[b];
    const int nn[3] = {B->nx, B->ny, B->nz};
    for (int f = 0; f < 6; ++f) {
      const or_face* F = &B->face[f];
      if (F->type < OR_PERIODIC || F->type > OR_OUTFLOW) return 11;
      if (f >= 4 && F->type != OR_PERIODIC) return 12;
      if (F->type != OR_INTERFACE) continue;
      if (F->nb < 0 || F->nb >= nb || F->nf < 0 || F->nf > 3) return 13;
      const or_block* B2 = &T->b[F->nb];
      const or_face* F2 = &B2->face[F->nf];
      if (F2->type != OR_INTERFACE || F2->nb != b || F2->nf != f || F2->rev != F->rev) return 14;
      const int n2[3] = {B2->nx, B2->ny, B2->nz};
      if (nn[1 - f / 2] != n2[1 - F->nf / 2]) return 15;
      if ((B->grid_xy == NULL) != (B2->grid_xy == NULL)) return 16;
      if (!B->grid_xy && (F->nf != (f ^ 1) || F->rev)) return 17;
      if ((nn[2] == 1) != (n2[2] == 1)) return 18;
    }
  }
  const int rr = p->order == 4 ? 2 : 1;
  for (int b = 0; b < nb; ++b) {
    const or_block* B = &T->b[b];
    or_term t[OR_MAXT];
    double cst[NV];
    for (int k = 0; k < B->nz; ++k)
      for (int j = -gmax; j < B->ny + gmax; ++j)
        for (int i = -gmax; i < B->nx + gmax; ++i) {
          const int di = i < 0 ? -i : (i >= B->nx ? i - B->nx + 1 : 0);
          const int dj = j < 0 ? -j : (j >= B->ny ? j - B->ny + 1 : 0);
          if (!di && !dj) continue;
          if (di && dj && (di > rr || dj > rr)) continue;  /* corners: viscous edges r x r only */
          if (resolve_state(T, b, i, j, k, t, cst) < 0) return 19;
        }
    T->M[b] = metric_plane(T, b);
  }
  return 0;
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
  if (p->compact) {
    /* Euler with the compact scheme of Eq. 2 (alpha = 1/3): R = -sum_a D_a F_a, D_a one
     * tridiagonal solve per owned line along a (or_compact_line), axes in the order x, y, z */
    const int sz3[3] = {d->sx, d->sy, d->sz};
    const int gz3[3] = {d->g, d->g, d->gz};
    const size_t no = (size_t)d->sx * d->sy * d->sz;
    for (size_t q = 0; q < NV * no; ++q) R[q] = 0.0;
    for (int a = 0; a < ndim; ++a) {
      const int na = sz3[a], a1 = (a + 1) % 3, a2 = (a + 2) % 3;
      double* fb = (double*)malloc(sizeof(double) * (size_t)(na + 8));
      double* db = (double*)malloc(sizeof(double) * (size_t)na);
      for (int t2 = 0; t2 < sz3[a2]; ++t2)
        for (int t1 = 0; t1 < sz3[a1]; ++t1)
          for (int vv = 0; vv < NV; ++vv) {
            const double* F = w->F + (size_t)a * NV * n + (size_t)vv * n;
            int c[3];
            c[a1] = t1;
            c[a2] = t2;
            for (int i = -4; i < na + 4; ++i) {
              c[a] = i;
              fb[i + 4] = F[(size_t)(c[0] + gz3[0]) + sty * (size_t)(c[1] + gz3[1]) + stz * (size_t)(c[2] + gz3[2])];
            }
            or_compact_line(na, h[a], fb, db);
            for (int i = 0; i < na; ++i) {
              c[a] = i;
              R[vv * no + (size_t)c[0] + (size_t)d->sx * ((size_t)c[1] + (size_t)d->sy * c[2])] -= db[i];
            }
          }
      free(fb);
      free(db);
    }
    return;
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
static void rhs_ext_curv(const or_params* p, const topo_t* T, const subdom* d, work_t* w, double* R) {
  const size_t ex = d->ex, ey = d->ey, ez = d->ez;
  const size_t n = ex * ey * ez;
  const size_t sty = ex, stz = ex * ey;
  const int three_d = p->nz > 1;
  const int ndim = three_d ? 3 : 2;
  const double gm = p->gamma, M2 = p->mach * p->mach;
  const int r = (p->order == 4) ? 2 : 1;
  double* E = w->E;
  double* W = w->W;
  double* Mx = w->M;
  /* metric terms at every extended point (from the block's extended metric plane) */
  for (int k = 0; k < (int)ez; ++k)
    for (int j = 0; j < (int)ey; ++j)
      for (int i = 0; i < (int)ex; ++i) {
        const int gx = d->ox + i - d->g, gy = d->oy + j - d->g;
        size_t q = (size_t)i + ex * (j + ey * (size_t)k);
        for (int c = 0; c < NM; ++c) Mx[c * n + q] = metric_at(T, d->b, c, gx, gy);
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

/* Block coordinates of extended point (i, j, k) of sub-domain d. */
static inline void ext_coord(const subdom* d, int i, int j, int k, int* c) {
  c[0] = d->ox + i - d->g;
  c[1] = d->oy + j - d->g;
  c[2] = d->oz + k - d->gz;
}

/* A halo source is the sub-domain's own value when it is reached without crossing a periodic
 * wrap or a block interface (a wall reflection or an outflow copy) and lies in the owned box;
 * every other source belongs to a neighbouring PE and is seen with the face's delay. */
static inline int term_own(const subdom* d, const or_term* t) {
  return !t->crossed && t->b == d->b && t->i >= d->ox && t->i < d->ox + d->sx && t->j >= d->oy &&
         t->j < d->oy + d->sy && t->k >= d->oz && t->k < d->oz + d->sz;
}

/* Delay of the foreign values at extended point (i, j, k): the face delay, or on an edge the
 * larger of the two faces' delays; faces on a physical boundary of the block carry none.
 * need = 0 for points the stencils never read. */
static int point_delay(const or_params* p, const subdom* d, int i, int j, int k, const int* kf, int* need) {
  int dep[3], face[3];
  int nout = classify(d, i, j, k, dep, face);
  const int r = (p->order == 4) ? 2 : 1;
  *need = 0;
  if (nout == 1) {
    *need = 1;
    for (int a = 0; a < 3; ++a)
      if (face[a] >= 0) return d->phys[face[a]] ? 0 : kf[face[a]];
  }
  if (nout == 2 && p->viscous) {
    int kd = 0;
    *need = 1;
    for (int a = 0; a < 3; ++a)
      if (face[a] >= 0) {
        if (dep[a] > r) *need = 0;
        if (!d->phys[face[a]] && kf[face[a]] > kd) kd = kf[face[a]];
      }
    return kd;
  }
  return 0;
}

/* Fill the extended array of sub-domain d for stage m-1 of step n.  Owned points and own halo
 * sources (wall mirror, outflow copy) take the current values, far-field points their state;
 * foreign sources by mode: 0 SA (the neighbour's current values), 1 AT (the halo buffer),
 * 2 AS (level n - k). */
static void fill_ext(const topo_t* T, const subdom* d, const double* Ucur, int mode, const hist_t* h, long n,
                     const int* kf, const halo_t* hb, work_t* w) {
  const or_params* p = &T->pb[d->b];
  const size_t ex = d->ex, ey = d->ey, ez = d->ez, ne = ex * ey * ez;
  for (size_t q = 0; q < NV * ne; ++q) w->E[q] = NAN;
  for (int k = 0; k < (int)ez; ++k)
    for (int j = 0; j < (int)ey; ++j)
      for (int i = 0; i < (int)ex; ++i) {
        int dep[3], face[3];
        const int nout = classify(d, i, j, k, dep, face);
        int need;
        const int kd = point_delay(p, d, i, j, k, kf, &need);
        if (nout != 0 && !need) continue;
        int c[3];
        ext_coord(d, i, j, k, c);
        const size_t q = (size_t)i + ex * (j + ey * k);
        if (nout == 0) {
          for (int v = 0; v < NV; ++v) w->E[v * ne + q] = Ucur[at_pt(T, d->b, v, c[0], c[1], c[2])];
          continue;
        }
        or_term t[OR_MAXT];
        double cst[NV];
        const int nt = resolve_state(T, d->b, c[0], c[1], c[2], t, cst);
        int foreign = 0;
        for (int m = 0; m < nt; ++m) foreign |= !term_own(d, &t[m]);
        for (int v = 0; v < NV; ++v) {
          double val = cst[v];
          for (int m = 0; m < nt; ++m) {
            const int own = term_own(d, &t[m]);
            if (own || mode == 0)
              val += t[m].w * refl_sign(v, t[m].flip) * Ucur[at_pt(T, t[m].b, v, t[m].i, t[m].j, t[m].k)];
            else if (mode == 2)
              val += t[m].w * refl_sign(v, t[m].flip) * H(h, n - kd)[at_pt(T, t[m].b, v, t[m].i, t[m].j, t[m].k)];
          }
          if (mode == 1 && foreign) val += hb->ub[v * ne + q];
          w->E[v * ne + q] = val;
        }
      }
}

/* Foreign part of a halo point from the delayed levels: sum over its foreign sources of
 * w s_v sum_l c_l U_v^{n-kd-l}. */
static double foreign_levels(const topo_t* T, const subdom* d, const or_term* t, int nt, int v, const hist_t* h,
                             long n, int kd, const double* c, int C) {
  double s = 0.0;
  for (int m = 0; m < nt; ++m) {
    if (term_own(d, &t[m])) continue;
    const size_t o = at_pt(T, t[m].b, v, t[m].i, t[m].j, t[m].k);
    double inner = 0.0;
    for (int l = 0; l < C; ++l) inner += c[l] * H(h, n - kd - l)[o];
    s += t[m].w * refl_sign(v, t[m].flip) * inner;
  }
  return s;
}

/* AT halo buffer: stage-0 extrapolation (Eq. 14/15), then buffer updates (Eq. 8, App. C). */
static void halo_init(const topo_t* T, const subdom* d, const hist_t* h, long n, const int* kf, halo_t* hb) {
  const or_params* p = &T->pb[d->b];
  const size_t ex = d->ex, ey = d->ey, ez = d->ez, ne = ex * ey * ez;
  const int C = or_levels(p->order);
  for (int k = 0; k < (int)ez; ++k)
    for (int j = 0; j < (int)ey; ++j)
      for (int i = 0; i < (int)ex; ++i) {
        int need;
        int kd = point_delay(p, d, i, j, k, kf, &need);
        if (!need) continue;
        double c[5];
        or_extrap_weights(p->order, (double)kd, c);
        int cc[3];
        ext_coord(d, i, j, k, cc);
        or_term t[OR_MAXT];
        double cst[NV];
        const int nt = resolve_state(T, d->b, cc[0], cc[1], cc[2], t, cst);
        size_t q = (size_t)i + ex * (j + ey * k);
        for (int v = 0; v < NV; ++v) {
          hb->ub[v * ne + q] = foreign_levels(T, d, t, nt, v, h, n, kd, c, C);
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


static void halo_update(const topo_t* T, const subdom* d, const hist_t* h, long n, const int* kf, int m,
                        const double* A, const double* B, halo_t* hb) {
  /* buffer update at stage m (1-based) uses the temporal derivative at stage e = m - 1 */
  const or_params* p = &T->pb[d->b];
  const size_t ex = d->ex, ey = d->ey, ez = d->ez, ne = ex * ey * ez;
  const int C = or_levels(p->order);
  for (int k = 0; k < (int)ez; ++k)
    for (int j = 0; j < (int)ey; ++j)
      for (int i = 0; i < (int)ex; ++i) {
        int need;
        int kd = point_delay(p, d, i, j, k, kf, &need);
        if (!need) continue;
        double dd[5];
        or_buffer_dudt(p->order, m - 1, (double)kd, dd);
        int cc[3];
        ext_coord(d, i, j, k, cc);
        or_term t[OR_MAXT];
        double cst[NV];
        const int nt = resolve_state(T, d->b, cc[0], cc[1], cc[2], t, cst);
        size_t q = (size_t)i + ex * (j + ey * k);
        for (int v = 0; v < NV; ++v) {
          const double s = foreign_levels(T, d, t, nt, v, h, n, kd, dd, C); /* = dt * dU/dt|_buf^(m-1) */
          double qn = A[m - 1] * hb->qb[v * ne + q] + s;
          hb->qb[v * ne + q] = qn;
          hb->ub[v * ne + q] += B[m - 1] * qn;
        }
      }
}

/* Wall point of block b: a point on a face of type wall (no-slip: its momentum is held at 0). */
static int wall_point(const topo_t* T, int b, int i, int j) {
  const or_block* B = &T->b[b];
  return (i == 0 && B->face[0].type == OR_WALL) || (i == B->nx - 1 && B->face[1].type == OR_WALL) ||
         (j == 0 && B->face[2].type == OR_WALL) || (j == B->ny - 1 && B->face[3].type == OR_WALL);
}

/* One filter pass along axis `ax` over all sub-domains: Uin -> Uout.  Window points beyond the
 * sub-domain: inside the block, the neighbour's value by the mode; beyond the block, the face's
 * sources (own ones current, foreign ones by the mode).  Wall points keep zero momentum. */
static void filter_pass(const topo_t* T, int ax, const double* Uin, double* Uout, int mode, const hist_t* h, long n,
                        int** kfs) {
  memcpy(Uout, Uin, sizeof(double) * NV * T->Ntot);
  const int nsub = T->nsub;
#pragma omp parallel for schedule(dynamic)
  for (int s = 0; s < nsub; ++s) {
    subdom d;
    make_sub(T, s, 0, &d);
    const or_params* p = &T->pb[d.b];
    if (ax == 2 && p->nz == 1) continue; /* two-dimensional block */
    const int C = or_levels(p->order);
    const int nn[3] = {p->nx, p->ny, p->nz};
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
            c[ax] = o[ax] + t;
            c[a1] = o[a1] + t1;
            c[a2] = o[a2] + t2;
            const int f = 2 * ax + (t < 0 ? 0 : 1);
            const int kd = d.phys[f] ? 0 : kf[f];
            double cw[5];
            if (mode == 1) or_extrap_weights(p->order, (double)(kd + 1), cw); /* to t_{n+1}: delay k + 1 */
            double val;
            if (t >= 0 && t < len) {
              val = Uin[at_pt(T, d.b, v, c[0], c[1], c[2])];
            } else if (c[ax] >= 0 && c[ax] < nn[ax]) {
              const size_t gq = at_pt(T, d.b, v, c[0], c[1], c[2]);
              if (mode == 0) val = Uin[gq];
              else if (mode == 2) val = H(h, n - kd)[gq];
              else {
                double sacc = 0.0;
                for (int l = 0; l < C; ++l) sacc += cw[l] * H(h, n - kd - l)[gq];
                val = sacc;
              }
            } else {
              or_term tt[OR_MAXT];
              double cst[NV];
              const int nt = resolve_state(T, d.b, c[0], c[1], c[2], tt, cst);
              val = cst[v];
              for (int m = 0; m < nt; ++m) {
                const size_t gq = at_pt(T, tt[m].b, v, tt[m].i, tt[m].j, tt[m].k);
                const double sg = tt[m].w * refl_sign(v, tt[m].flip);
                if (mode == 0 || term_own(&d, &tt[m])) val += sg * Uin[gq];
                else if (mode == 2) val += sg * H(h, n - kd)[gq];
                else {
                  double sacc = 0.0;
                  for (int l = 0; l < C; ++l) sacc += cw[l] * H(h, n - kd - l)[gq];
                  val += sg * sacc;
                }
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
            const int zero = v >= 1 && v <= 3 && wall_point(T, d.b, c[0], c[1]);
            Uout[at_pt(T, d.b, v, c[0], c[1], c[2])] = zero ? 0.0 : out[t];
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

/* Volume-averaged kinetic energy and enstrophy (Sec. 5.2, rho_0 = 1) with vorticity from the CD
 * scheme, cell-volume-weighted totals of the conserved variables, and a non-finite flag, over
 * all blocks.  out[8] = {K, eps, sum rho, sum rho u, sum rho v, sum rho w, sum rho E, nan}.
 * On a curvilinear block the cell volume is J^-1 and the averages are volume-weighted; velocity
 * derivatives are taken in index space and mapped by the metric terms.  The enstrophy average
 * covers the points whose CD stencils stay inside their block or cross only periodic faces. */
static void diag_topo(const topo_t* T, const double* U, double* out) {
  double ke = 0, ens = 0, vol = 0, vole = 0, tot[5] = {0, 0, 0, 0, 0};
  int bad = 0;
  /* averaging weights: cell volumes in units of the first Cartesian block's cell */
  double dVref = 1.0;
  for (int b = T->nb - 1; b >= 0; --b)
    if (!T->M[b]) dVref = T->pb[b].dx * T->pb[b].dy * (T->pb[b].nz > 1 ? T->pb[b].dz : 1.0);
  for (int b = 0; b < T->nb; ++b) {
    const or_params* p = &T->pb[b];
    const or_block* B = &T->b[b];
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    const int curv = T->M[b] != NULL;
    const double dV0 = p->dx * p->dy * (nz > 1 ? p->dz : 1.0);
    const int order = p->order, rs = order == 4 ? 2 : 1;
    const int nn[3] = {nx, ny, nz};
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
          const double dV = curv ? metric_at(T, b, 5, i, j) : dV0;
          const int c0[3] = {i, j, k};
          double rho = U[at_pt(T, b, 0, i, j, k)];
          double u = U[at_pt(T, b, 1, i, j, k)] / rho, v = U[at_pt(T, b, 2, i, j, k)] / rho;
          double w = U[at_pt(T, b, 3, i, j, k)] / rho;
          for (int c = 0; c < 5; ++c) {
            const double x = U[at_pt(T, b, c, i, j, k)];
            if (!isfinite(x)) bad = 1;
            tot[c] += x * dV;
          }
          const double wv = dV / dVref; /* volume-weighted averages (a point average on one uniform block) */
          vol += wv;
          ke += 0.5 * rho * (u * u + v * v + w * w) * wv;
          int inner = 1;
          for (int a = 0; a < 3; ++a)
            if (nn[a] > 1 && (c0[a] < rs && B->face[2 * a].type != OR_PERIODIC)) inner = 0;
            else if (nn[a] > 1 && (c0[a] > nn[a] - 1 - rs && B->face[2 * a + 1].type != OR_PERIODIC)) inner = 0;
          if (!inner) continue;
          /* velocity derivative along axis a of component c at (i,j,k), periodic CD */
          double dvel[3][3];
          for (int c = 0; c < 3; ++c)
            for (int a = 0; a < 3; ++a) {
              int n_a = nn[a];
              if (n_a == 1) { dvel[c][a] = 0.0; continue; }
              double hh = curv ? 1.0 : (a == 0 ? p->dx : (a == 1 ? p->dy : p->dz));
              double f[5];
              for (int o = -2; o <= 2; ++o) {
                if (rs == 1 && (o == -2 || o == 2)) { f[o + 2] = 0.0; continue; }
                int ii = i, jj = j, kk = k;
                if (a == 0) ii = wrapi(i + o, nx);
                if (a == 1) jj = wrapi(j + o, ny);
                if (a == 2) kk = wrapi(k + o, nz);
                f[o + 2] = U[at_pt(T, b, 1 + c, ii, jj, kk)] / U[at_pt(T, b, 0, ii, jj, kk)];
              }
              if (order == 4)
                dvel[c][a] = ((-1.0 / 3.0) * (f[4] - f[0]) / 4.0 + (4.0 / 3.0) * (f[3] - f[1]) / 2.0) / hh;
              else
                dvel[c][a] = (f[3] - f[1]) / (2.0 * hh);
            }
          if (curv) {
            /* d u_c / d x_j = J sum_a (metric row a)_j d u_c / d xi_a */
            const double J = 1.0 / dV;
            const double m[3][3] = {{metric_at(T, b, 0, i, j), metric_at(T, b, 1, i, j), 0.0},
                                    {metric_at(T, b, 2, i, j), metric_at(T, b, 3, i, j), 0.0},
                                    {0.0, 0.0, metric_at(T, b, 4, i, j)}};
            double dphys[3][3];
            for (int c = 0; c < 3; ++c)
              for (int jj = 0; jj < 3; ++jj)
                dphys[c][jj] = J * (m[0][jj] * dvel[c][0] + m[1][jj] * dvel[c][1] + m[2][jj] * dvel[c][2]);
            memcpy(dvel, dphys, sizeof(dvel));
          }
          double wx = dvel[2][1] - dvel[1][2], wy = dvel[0][2] - dvel[2][0], wz = dvel[1][0] - dvel[0][1];
          ens += 0.5 * rho * (wx * wx + wy * wy + wz * wz) * wv;
          vole += wv;
        }
  }
  out[0] = ke / vol;
  out[1] = vole > 0 ? ens / vole : 0.0;
  for (int c = 0; c < 5; ++c) out[2 + c] = tot[c];
  out[7] = bad ? 1.0 : 0.0;
}

int or_diagnostics(const or_params* p, const double* U, double* out) {
  topo_t T;
  const int g = halo_g(p);
  int rc = topo_build(p, g, g, &T);
  if (rc == 0) diag_topo(&T, U, out);
  topo_free(&T);
  return rc;
}

/* Initial-history state for a resumed run: levels n0 - R + 1 .. n0 may be passed in `hist_in`
 * ([R][5][N], level n0 - R + 1 first); NULL means a fresh start at n0 = 0 from U0. */

/*
 * Advance `nsteps` steps starting from step index n0 with state U (in/out; all blocks, block
 * after block).
 * delays: SAA table int8 [n0 + nsteps][nsub][6] (ignored for SA/CAA).
 * diag (optional): per step [nsteps][8] = KE, enstrophy, sum rho, sum rho u, sum rho v,
 *                  sum rho w, sum rho E, nan-flag (after the step).
 * Returns 0 on success, nonzero on invalid input.
 */
int or_run(const or_params* p, double* U, const int8_t* delays, long n0, long nsteps, const double* hist_in,
           double* diag) {
  const int C = or_levels(p->order);
  const int g = halo_g(p);
  double A[5], B[5];
  const int S = or_lserk(p->order, A, B);
  const int need = g > (p->filter ? 5 : 0) ? g : (p->filter ? 5 : 0);
  topo_t T;
  int rc = topo_build(p, g, need, &T);
  if (rc) { topo_free(&T); return rc; }
  if (p->mlp && p->nblocks > 0) { topo_free(&T); return 20; }
  if (p->compact && (p->viscous || p->order != 4 || p->nblocks > 0 || p->grid_xy || p->mlp)) { topo_free(&T); return 24; }
  const size_t NT = T.Ntot;
  const int nsub = T.nsub;
  /* validation: every sub-domain at least as wide as the halo it needs */
  for (int s = 0; s < nsub; ++s) {
    subdom d;
    make_sub(&T, s, g, &d);
    if (d.sx < need || d.sy < need || (T.pb[d.b].nz > 1 && d.sz < need)) { topo_free(&T); return 1; }
  }
  if (p->algo == 1 && p->caa_L < 1) { topo_free(&T); return 2; }
  hist_t h;
  h.R = ring_depth(p);
  h.lev = (double**)malloc(sizeof(double*) * h.R);
  for (int i = 0; i < h.R; ++i) h.lev[i] = (double*)calloc(NV * NT, sizeof(double));
  if (hist_in) {
    for (int i = 0; i < h.R; ++i) {
      long lvl = n0 - h.R + 1 + i;
      if (lvl >= 0) memcpy(h.lev[lvl % h.R], hist_in + (size_t)i * NV * NT, sizeof(double) * NV * NT);
    }
  }
  memcpy(h.lev[n0 % h.R], U, sizeof(double) * NV * NT);

  double* Ucur = (double*)malloc(sizeof(double) * NV * NT);
  double* Unew = (double*)malloc(sizeof(double) * NV * NT);
  double* Q = (double*)malloc(sizeof(double) * NV * NT);
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
    memcpy(Ucur, H(&h, n), sizeof(double) * NV * NT);
    memset(Q, 0, sizeof(double) * NV * NT);
    for (int m = 1; m <= S; ++m) {
#pragma omp parallel
      {
        work_t w;
        memset(&w, 0, sizeof(w));
#pragma omp for schedule(dynamic)
        for (int s = 0; s < nsub; ++s) {
          subdom d;
          make_sub(&T, s, g, &d);
          const or_params* pb = &T.pb[d.b];
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
              halo_init(&T, &d, &h, n, kfs[s], &hbs[s]);
              if (p->mlp) halo_init_learned(pb, &d, s, &h, n, kfs[s], &hbs[s]);
            }
          }
          fill_ext(&T, &d, Ucur, mode, &h, n, kfs[s], &hbs[s], &w);
          size_t no = (size_t)d.sx * d.sy * d.sz;
          double* R = (double*)malloc(sizeof(double) * NV * no);
          if (T.M[d.b]) rhs_ext_curv(pb, &T, &d, &w, R);
          else rhs_ext(pb, &d, &w, R);
          /* Eq. 3: Q^(m) = A_m Q^(m-1) + dt R(U^(m-1));  U^(m) = U^(m-1) + B_m Q^(m); no-slip
           * wall points keep zero momentum */
          for (int v = 0; v < NV; ++v)
            for (int k = 0; k < d.sz; ++k)
              for (int j = 0; j < d.sy; ++j)
                for (int i = 0; i < d.sx; ++i) {
                  size_t gq = at_pt(&T, d.b, v, d.ox + i, d.oy + j, d.oz + k);
                  size_t o = (size_t)i + (size_t)d.sx * (j + (size_t)d.sy * k);
                  double qn = A[m - 1] * Q[gq] + p->dt * R[v * no + o];
                  double un = Ucur[gq] + B[m - 1] * qn;
                  if (v >= 1 && v <= 3 && wall_point(&T, d.b, d.ox + i, d.oy + j)) qn = un = 0.0;
                  Q[gq] = qn;
                  Unew[gq] = un;
                }
          free(R);
          if (mode == 1 && m <= S - 1) halo_update(&T, &d, &h, n, kfs[s], m, A, B, &hbs[s]);
        }
        work_free(&w);
      }
      double* t = Ucur; Ucur = Unew; Unew = t;
    }
    if (p->filter) {
      for (int ax = 0; ax < 3; ++ax) {
        filter_pass(&T, ax, Ucur, Unew, mode, &h, n, kfs);
        double* t = Ucur; Ucur = Unew; Unew = t;
      }
    }
    memcpy(h.lev[(n + 1) % h.R], Ucur, sizeof(double) * NV * NT);
    if (diag) diag_topo(&T, Ucur, diag + (size_t)(n - n0) * 8);
  }
  memcpy(U, Ucur, sizeof(double) * NV * NT);
  for (int i = 0; i < h.R; ++i) free(h.lev[i]);
  free(h.lev);
  free(Ucur); free(Unew); free(Q);
  for (int s = 0; s < nsub; ++s) { free(kfs[s]); free(hbs[s].ub); free(hbs[s].qb); }
  free(kfs); free(hbs);
  topo_free(&T);
  return 0;
}

/* R(U) of all blocks in synchronous mode (halos = current neighbour values or the boundary
 * sources). */
int or_rhs(const or_params* p, const double* U, double* Rout) {
  const int g = halo_g(p);
  if (p->compact && (p->viscous || p->order != 4 || p->nblocks > 0 || p->grid_xy)) return 24;
  int kf[6] = {0, 0, 0, 0, 0, 0};
  topo_t T;
  int rc = topo_build(p, g, g, &T);
  if (rc) { topo_free(&T); return rc; }
  for (int s = 0; s < T.nsub; ++s) {
    subdom d;
    make_sub(&T, s, g, &d);
    if (d.sx < g || d.sy < g || (T.pb[d.b].nz > 1 && d.sz < g)) { topo_free(&T); return 1; }
  }
#pragma omp parallel
  {
    work_t w;
    memset(&w, 0, sizeof(w));
#pragma omp for schedule(dynamic)
    for (int s = 0; s < T.nsub; ++s) {
      subdom d;
      make_sub(&T, s, g, &d);
      const or_params* pb = &T.pb[d.b];
      work_reserve(&w, (size_t)d.ex * d.ey * d.ez);
      fill_ext(&T, &d, U, 0, NULL, 0, kf, NULL, &w);
      size_t no = (size_t)d.sx * d.sy * d.sz;
      double* R = (double*)malloc(sizeof(double) * NV * no);
      if (T.M[d.b]) rhs_ext_curv(pb, &T, &d, &w, R);
      else rhs_ext(pb, &d, &w, R);
      for (int v = 0; v < NV; ++v)
        for (int k = 0; k < d.sz; ++k)
          for (int j = 0; j < d.sy; ++j)
            for (int i = 0; i < d.sx; ++i)
              Rout[at_pt(&T, d.b, v, d.ox + i, d.oy + j, d.oz + k)] =
                  R[v * no + (size_t)i + (size_t)d.sx * (j + (size_t)d.sy * k)];
      free(R);
    }
    work_free(&w);
  }
  topo_free(&T);
  return 0;
}

/* Sources of the points ijk[npts][3] of block b (beyond its faces) as the oracle resolves them,
 * for cross-checking another implementation: per point 34 values -- count, far-field constant
 * [5], then per source block, i, j, k, weight, mirrored, crossed (7 values, up to OR_MAXT
 * sources).  Returns nonzero for an invalid description or a point that does not resolve. */
int or_halo_sources(const or_params* p, int b, long npts, const int* ijk, double* outs) {
  const int g = halo_g(p);
  topo_t T;
  int rc = topo_build(p, g, g, &T);
  if (rc == 0 && (b < 0 || b >= T.nb)) rc = 21;
  for (long q = 0; rc == 0 && q < npts; ++q) {
    const int i = ijk[3 * q], j = ijk[3 * q + 1], k = ijk[3 * q + 2];
    double* out = outs + 34 * q;
    or_term t[OR_MAXT];
    double cst[NV];
    const int n = resolve_state(&T, b, i, j, k, t, cst);
    if (n < 0) rc = 22;
    else {
      out[0] = n;
      for (int v = 0; v < NV; ++v) out[1 + v] = cst[v];
      for (int m = 0; m < OR_MAXT; ++m) {
        double* o = out + 6 + 7 * m;
        if (m >= n) { for (int q = 0; q < 7; ++q) o[q] = 0.0; continue; }
        o[0] = t[m].b; o[1] = t[m].i; o[2] = t[m].j; o[3] = t[m].k;
        o[4] = t[m].w; o[5] = t[m].flip; o[6] = t[m].crossed;
      }
    }
  }
  topo_free(&T);
  return rc;
}

/* Metric terms {xi^_x, xi^_y, eta^_x, eta^_y, zeta^_z, J^-1} at the points ij[npts][2] of curvilinear
 * block b's extended plane, as the oracle computes them (for cross-checking another
 * implementation); out[npts][6].  Returns nonzero for an invalid description or a Cartesian block. */
int or_metric_terms(const or_params* p, int b, long npts, const int* ij, double* out) {
  const int g = halo_g(p);
  topo_t T;
  int rc = topo_build(p, g, g, &T);
  if (rc == 0 && (b < 0 || b >= T.nb || !T.M[b])) rc = 23;
  for (long q = 0; rc == 0 && q < npts; ++q)
    for (int c = 0; c < NM; ++c) out[NM * q + c] = metric_at(&T, b, c, ij[2 * q], ij[2 * q + 1]);
  topo_free(&T);
  return rc;
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
