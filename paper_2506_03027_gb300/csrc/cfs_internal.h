// cfs_internal.h -- library-private declarations shared by the host (capi.cpp, coeffs.cpp) and
// the CUDA translation units of libcfs.  Not part of the public C ABI (include/cfs.h).
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#define CFS_MAX_DELAY 15   // largest supported delay k (ring depth <= 15 + 5 + 1)
#define CFS_MAX_LEVELS 5   // C: delayed levels of AT4
#define CFS_MAX_STAGES 5   // s: stages of LSERK4
#define CFS_MAX_LINE 128   // longest sub-domain line of the compact scheme

// learned halo predictor: one face column of HDEPTH halo points, 5 variables
#define MLP_HDEPTH 4
#define MLP_KMAX 4                                   // delays 0..4 (one-hot)
#define MLP_NIN (3 * MLP_HDEPTH * 5 + MLP_KMAX + 1)  // 65
#define MLP_NH 64
#define MLP_NOUT (MLP_HDEPTH * 5)                    // 20
// the solver's feature tiles: 128 face columns x 72 inputs (65 padded to a multiple of 8), FP32
#define MLP_TILE 128
#define MLP_K1 72
#define MLP_OFF_W1 0
#define MLP_OFF_B1 (MLP_OFF_W1 + MLP_NH * MLP_NIN)
#define MLP_OFF_W2 (MLP_OFF_B1 + MLP_NH)
#define MLP_OFF_B2 (MLP_OFF_W2 + MLP_NH * MLP_NH)
#define MLP_OFF_W3 (MLP_OFF_B2 + MLP_NH)
#define MLP_OFF_B3 (MLP_OFF_W3 + MLP_NOUT * MLP_NH)
#define MLP_NPARAM (MLP_OFF_B3 + MLP_NOUT)           // 9684

namespace cfs {

// Sub-domain descriptor (one per processing element of Sec. 3).
struct SubDev {
  int ox, oy, oz;     // owned box origin (global point indices)
  int sx, sy, sz;     // owned box size
  int ex, ey, ez;     // padded ("view") box size: owned + halo G (Gz = 0 in 2-D)
  int ix, iy, iz;     // sub-domain coordinates in the decomposition grid
  long long pbase;    // offset of the padded box in the scratch arrays (points)
  // the block the sub-domain belongs to (each block periodic in itself)
  int bnx, bny, bnz;  // block size
  long long bN;       // block points
  long long bbase;    // offset of the block's state [5][bnz][bny][bnx] in a state array (doubles)
  double c1[3], c2[3];  // CD coefficients of the block's spacing: c1 = (a/2)/h, c2 = (b/4)/h
  // curvilinear block: offset of its metric plane in Geometry::metric, -1 for a uniform Cartesian
  // block (c1, c2 are then the index-space coefficients, h = 1).  The plane covers the block's
  // (x, y) points extended by G on every side, row length mx, component stride mpl; it is the
  // same for every z (blocks are extruded)
  long long mbase;
  int mx;
  long long mpl;
  // faces of the sub-domain on a physical boundary of the block (bit f, faces -x, +x, -y, +y,
  // -z, +z) and, among them, the no-slip walls
  int phys, wall;
  // block with a non-periodic face: offset of its gather map in Geometry::emap (an entry index,
  // or -1, for every point of the block's (x, y) range extended by GE, all z: row length gmx,
  // plane gmx * gmy); -1 for a block periodic on every face
  long long ebase;
  int gmx, gmy;
  // 1: this context computes the sub-domain; 0: another process owns it (a partitioned context,
  // cfs_set_partition): its points are neither updated nor read here except through the strips
  // the exchange delivers
  int own;
};

// Sources of the state at a point beyond a non-periodic block face (an interface, a wall mirror,
// an outflow copy, a far field): U_v = cst_v + sum_t w_t s_v(t) U_v(source t), s_v = -1 for the
// momentum of a mirrored source.  A source is the receiving sub-domain's own value when it was
// reached without crossing a periodic wrap or an interface and lies in that sub-domain.
struct GatherEntry {
  long long off[4];  // source: state offset of its block plus its point index (component v at + v bN)
  double w[4];
  double cst[5];
  int bN[4];         // source block's points
  int sid[4];        // sub-domain owning the source
  int flags[4];      // bit 0: momentum negated; bit 1: crossed a periodic wrap or an interface
  int nt;
  int pad;
};
#define GATHER_MAXT 4

// Scalars every kernel needs; passed by value.
struct Geometry {
  int nx, ny, nz;        // size of the first block (single-block runs: the grid)
  long long N;           // points of all blocks (a state array holds 5 N doubles)
  int nsub;              // number of sub-domains
  int G, Gz;             // halo depth in x/y and in z
  int r;                 // stencil radius (2 for CD4, 1 for CD2)
  int ndim;              // 2 or 3
  int viscous;
  long long Ptot;        // total padded points (scratch length per component)
  // metric planes of the curvilinear blocks, [NMETRIC][mpl] per block (device), or null:
  // xi^_x, xi^_y, eta^_x, eta^_y, zeta^_z (= J^-1 d(xi,eta,zeta)/dx of App. A), J^-1, J
  const double* metric;
  // gather maps and entries of the blocks with non-periodic faces (device), or null
  const int* emap;
  const GatherEntry* gent;
  int GE;                // depth of the gather maps beyond the block faces
  int fs;                // depth of the flux strips beyond each face: r, or 4 for the compact scheme
};
#define NMETRIC 7

struct Physics {
  double gamma, gm1, gM2;  // gamma, gamma - 1, gamma M^2
  double ire;              // 1 / Re
  double kappa;            // 1 / ((gamma - 1) Pr M^2)
  // the primitives' temperature slot holds kappa T (the heat flux is then its plain gradient):
  // kgM2 = kappa gamma M^2; ivT = 1/Re, times kappa^-a for the power law (its mu = T^a is taken as
  // (kappa T)^a kappa^-a)
  double kgM2, ivT;
  int visc_law;
  double visc_exp;
  double c1[3], c2[3];     // CD coefficients per axis: c1 = (a/2)/h, c2 = (b/4)/h
  // FP32-intermediate form only: reference pressure p_ref = 1/(gamma M^2), E_ref = p_ref/(gamma-1)
  // and H_ref = E_ref + p_ref; primitives carry p - p_ref and rho E - E_ref so that FP32 rounding
  // acts on O(1) deviations instead of p ~ 1/(gamma M^2)
  double p_ref, E_ref, H_ref;
};

// Delay schedule as seen by the kernels of one step.
struct StepSched {
  int mode;              // 0 SA (halo = live neighbour), 1 AT, 2 AS
  long long n;           // step index
  int R;                 // ring depth
  int algo;              // 0 SA, 1 CAA, 2 SAA
  int L;                 // CAA interval
  int C;                 // delayed levels
  long long cap;         // clamp: k <= n - C + 1
  const int8_t* table;   // SAA delays of this step [nsub][6] (device), or null
  const double* W;       // device: AT halo weights [(k * s + m) * C + l]
  const float* W32;      // device: the same table for sums over level differences as pairs of floats
                         // (hi, lo) per entry: entry l = 0 holds sum_l W - 1, entries l >= 1 W_l
  const float* W32d;     // device: as W32 for the differences W^(m) - W^(0) (learned face halos)
  const double* LH;      // device: learned stage-0 face-halo values [5][Ptot], or null (plain AT)
  const double* Wf;      // device: filter-halo extrapolation weights c(k+1) [k * C + l]
  // CUDA-graph mode: the step index lives in device memory (dn); kernels derive n, mode, cap and
  // the SAA table row from it, so one captured step serves every step
  const long long* dn;
  int at;                // 1: AT, 0: AS (for the mode derived from dn)
  int nsub;
  const int8_t* table_base;
  long long Ntot;        // points of a state array (ring level stride / 5)
  int* status;           // device: bit 0 set by a bounded wait that gave up (read as CFS_ETIMEOUT), or null
};

// coefficient generation (coeffs.cpp)
int lserk_coeffs(int order, double* A, double* B);
bool extrap_weights(int order, int k, long double* c);
bool buffer_dudt_weights(int order, int e, int k, long double* d);
int at_weight_table(int order, int kmax, double* W);
int filter_extrap_table(int order, int kmax, double* Wf);
bool pade10_coeffs(double alpha, double* a);
// Block topology (host): faces of the connected multi-block grid.
enum { FACE_PERIODIC = 0, FACE_INTERFACE = 1, FACE_WALL = 2, FACE_FARFIELD = 3, FACE_OUTFLOW = 4 };
struct FaceSpec {
  int type = FACE_PERIODIC;
  int nb = -1, nf = -1, rev = 0;
  double state[5] = {0, 0, 0, 0, 0};
  double shift[2] = {0, 0};
};
struct TopoBlock {
  int n[3];
  int P[3];
  int sid0;
  long long base, N;
  const double* xy;  // curvilinear: [2][ny][nx], or null
  double shift[4];
  FaceSpec face[6];
};
// topology.cpp
const char* topo_check(const TopoBlock* B, int nb);  // null when valid, else the reason
bool topo_periodic(const TopoBlock& b);
// Sources of point (i, j, k) of block b's index space, for inspection: out[0] = count, out[1..5]
// the far-field constant, then per source (up to 4) block, i, j, k, weight, mirrored, crossed.
int halo_sources(const TopoBlock* B, int nb, int b, int i, int j, int k, double* out);
// Gather entry of point (i, j, k) of block b's index space; false if it does not resolve.
bool gather_entry(const TopoBlock* B, int nb, int b, int i, int j, int k, GatherEntry* e);
// Metric plane [NMETRIC][(nx + 2G)(ny + 2G)] of curvilinear block b; false if the grid does not
// continue far enough across a face, or a cell volume is not positive.
bool metric_plane(const TopoBlock* B, int nb, int b, int G, int r, int order, double dz, int ndim, double* M);

// kernel launchers (kernels.cu); all return a cudaError_t cast to int

struct StageLaunch {
  const double* Uin;
  double* Uout;
  double* Q;
  const double* ring;   // [R][5][N]
  const SubDev* subs;   // device table
  void* Wp;             // scratch [7][Ptot] primitives, in the intermediate precision
  void* Phi;            // scratch [15][Ptot] combined fluxes, in the intermediate precision
  int stage;            // 0-based stage index m-1 (selects the halo weights W^(m-1))
  int s;                // number of stages
  double A, B, dt;
  int first, last;      // first stage skips reading Q, last stage skips writing Q
  int in_ring, out_ring;  // graph mode: input is ring level n / output is ring level n + 1
  int threads;          // threads per CTA (128, 256 or 512)
  int max_pad;          // largest padded box (points)
  const int* halo;      // device: (sub-domain, padded index) pairs of every halo point
  long long nhalo;
  int max_own;          // largest owned box (points)
  int max_flux;         // largest flux region box (points)
  // compact scheme (Eq. 2, alpha = 1/3): the flux divergence by line solves into R ([5][N], FP64),
  // then the stage update from R; cthomas = [Lmax + 1 rows][2][Lmax] Thomas factors per line
  // length (forward factor c'_i, reciprocal pivot 1 / m_i)
  int compact;
  double* R;
  const double* cthomas;
  int Lmax;
};

// Optional per-kernel event timing: when non-null, the launchers call rec(kind, begin) around
// every kernel on the launch stream.
struct Timer {
  void (*rec)(void* self, int kind, int begin);
  void* self;
};

int launch_stage(const Geometry& g, const Physics& ph, const StepSched& sc, const StageLaunch& a,
                 int precision, void* stream, long long* launches, const Timer* tm);

struct FilterLaunch {
  long long ebase;         // the block's gather map (SubDev::ebase), or -1
  int gmx, gmy;
  int wall;                // bit f: face f of the block is a no-slip wall (momentum held at zero)
  int phys;                // bit f: face f of the block is a physical boundary
  const double* Uin;
  double* Uout;
  const double* ring;
  int nx, ny, nz;          // the block being filtered
  long long bN, bbase;     // its points and the offset of its state in a state array
  int sid0;                // index of its first sub-domain
  int in_ring, out_ring;   // graph mode: input is ring level n / output is ring level n + 1
  const int* owner[3];     // device: sub-domain index along each axis for every global coordinate
  const int* axis_off[3];  // device: per sub-domain index along the axis, its origin
  const int* axis_len[3];  // device: ... and its length
  const double* thomas;    // device: [Lmax+1 rows][2][Lmax] Thomas factors per line length
  const float* thomas32;   // device: the same table rounded to FP32 (d2f_fast), for the FP32 form
  int Lmax;
  int Lt;                  // longest sub-domain line of this block along the pass axis (sizes the tiles)
  int P[3];                // sub-domains per axis
  double alpha;
  double h[6];             // filter right side: a_0, a_1/2, ..., a_5/2
  double b1;               // a_1/2 - alpha: weight of the first second difference (increment form)
  int only_sync;           // graph mode beside the sub-domain filter: return unless the step is synchronous
  const SubDev* subs;      // partitioned context: the sub-domain table (lines of foreign sub-domains are
                           // skipped); null when every sub-domain is computed here
};

// FP32-intermediate filter of asynchronous steps, all three passes per (sub-domain, variable)
// (filter_block.cu); cubic sub-domains of n points per axis, n in {16, 32}.
struct FilterBlockLaunch {
  const double* Uin;
  double* Uout;
  const double* ring;
  int in_ring, out_ring;
  const SubDev* subs;
  int nsub;
  const double* thomas;
  int Lmax;
  double alpha;
  double h[6];
  double b1;
  // the passes' halos as FP32 deviations from the (sub-domain, variable) reference value,
  // [nsub * 5][3 axes][10][N * N], written by k_filter_block_halo
  float* halo;
};
bool filter_block_supported(int n);
int launch_filter_block(const Geometry& g, const StepSched& sc, const FilterBlockLaunch& f, int n, void* stream,
                        long long* launches, const Timer* tm);

int filter_prepare(int Lmax, int precision);
int launch_round_table(const double* x, float* y, long long n, void* stream);  // y = d2f_fast(x)  // shared-memory attribute of the filter kernels; nonzero if too long
int launch_filter(const Geometry& g, const StepSched& sc, const FilterLaunch& f, int axis, int precision,
                  void* stream, long long* launches, const Timer* tm);

// Fused stage for the FP32-intermediate form (fused.cu): 3-D Navier-Stokes, CD4/AT4.
struct FusedLaunch {
  const double* Uin;
  double* Uout;
  double* Q;
  const SubDev* subs;
  const int* work;      // device: 4 ints per tile (sub-domain, x0, y0, z0 | z1 << 16)
  int nwork;
  int grid;             // persistent grid size
  int fy;               // tile height: 4, 8 or 16 (tile width 32)
  const float* Wh;      // per-step AT/AS halo primitives [s][7][Ptot]
  int stage;
  double A, B, dt;
  int first, last;
  const double* ring;
  int in_ring, out_ring;
  int curv;             // 1: the context has curvilinear blocks (metric window in shared memory)
};
int fused_smem_bytes(int fy, int curv);
int fused_blocks_per_sm(int fy, int curv, int* blocks);  // sets the shared-memory attribute, then asks the occupancy API
int launch_halo_prims(const Geometry& g, const Physics& ph, const StepSched& sc, const double* ring, const SubDev* subs,
                      const int* halo, long long nhalo, float* Wh, int s, void* stream, long long* launches,
                      const Timer* tm);
int launch_stage_fused(const Geometry& g, const Physics& ph, const StepSched& sc, const FusedLaunch& a, void* stream,
                       long long* launches, const Timer* tm);

// learned halo network (mlp.cu)
size_t mlp_smem_bytes();
long long mlp_workspace_floats(long long nsamp);
int launch_mlp_forward(const float* params, const void* x_bf16, float* y, long long nsamp, void* stream);
int launch_mlp_grad(const float* params, const void* x_bf16, const float* target, long long nsamp, float* workspace,
                    float* grad, float* loss, void* stream);
int launch_adamw(float* params, const float* grad, float* m, float* v, int n, int step, float lr, float b1, float b2,
                 float eps, float wd, void* stream);
// feature scales: in_scale[5] (delayed-level differences), own_scale[5], out_scale[5]
struct MlpScales {
  double in[5], own[5], out[5];
};
// Samples for training: spec[i] = (sub-domain, face, t1, t2, k); features from levels n-k..n-k-2 of
// the ring (halo) and n, n-k (own), target = (U^n - 3-level extrapolation) * out scale.
// at4 (or null): the residual of the AT4 stage-0 value (5 levels, weights sc.W of s stages) likewise.
int launch_halo_samples(const Geometry& g, const StepSched& sc, const double* ring, const SubDev* subs, const int* spec,
                        long long n, MlpScales sc_, void* x_bf16, float* target, float* at4, int s, void* stream);
// Solver: stage-0 halo values of every face column from the network (AT mode), into LH[5][Ptot].
int launch_mlp_halo(const Geometry& g, const StepSched& sc, const double* ring, const SubDev* subs, const int* cols,
                    long long ncol, const float* params, MlpScales sc_, float* X, double* A3, double* LH, void* stream, long long* launches,
                    const Timer* tm);

// Diagnostics over all blocks: per block (size, state offset, CD coefficients, cell volume) the
// block partial sums go to rows [row0, row0 + nblocks) of partial; the final pass reduces nrows.
struct DiagBlock {
  int nx, ny, nz;
  long long bN, bbase;
  double c1[3], c2[3], dV;
  const double* M;  // the block's metric plane (curvilinear), or null
  int mx, G;        // its row length and extension
  long long mpl;    // its component stride
  int nonper;       // bit f: face f is not periodic (no enstrophy within the stencil radius of it)
  int rs;           // stencil radius
  // partitioned context: only the points of sub-domains computed here count (owner[a][coordinate]
  // = sub-domain index along axis a, P the split, sid0 the block's first sub-domain); subs null
  // when every sub-domain is computed here
  const SubDev* subs;
  const int* owner[3];
  int P[3], sid0;
};
#define DIAG_NQ 9   // per block row: K, enstrophy, 5 totals, non-finite flag, enstrophy volume
int launch_diagnostics_block(const Geometry& g, const DiagBlock& b, const double* U, double* partial, int row0,
                             int nblocks, void* stream);
int launch_diagnostics_final(const double* partial, int nrows, double* out, double volume, void* stream);
int launch_advance_step(long long* dn, void* stream);
int launch_eval_power(const double* x, double a, double* y, long long n, void* stream);
int launch_fp64_probe(double* sink, int blocks, int iters, void* stream);
// Self-test of the bounded device waits: one CTA waits on an mbarrier that nothing arrives at, gives
// up after `limit` polls and sets bit 0 of *status.
int launch_wait_check(int* status, unsigned limit, void* stream);
// Strip exchange of a partitioned context: buf[5 i + v] = U[off[i] + v bN[i]] (pack) and the
// reverse (unpack) for the n entries of a plan.
int launch_strip_pack(const double* U, const long long* off, const int* bN, long long n, double* buf, void* stream);
int launch_strip_unpack(double* U, const long long* off, const int* bN, long long n, const double* buf, void* stream);

// Exchange plan of a partitioned context (partition.cpp): for this rank and every peer q, the state
// offsets (block base + point index; component v at + v x the block's points) of the points it
// sends to q -- its own points that q's sub-domains read -- and of those it receives from q,
// both sorted, so that rank p's send list to q is rank q's receive list from p.  The read set of
// a sub-domain: faces to depth `depth` (x, y; z to depth_z), viscous edges to r x r.
struct StripPlan {
  std::vector<long long> send_off, recv_off;  // [nranks + 1] prefix offsets into the lists (points)
  std::vector<long long> send, recv;          // state offsets
  std::vector<int> send_bN, recv_bN;          // points of the entry's block
};
const char* strip_plan(const TopoBlock* B, int nb, int nsub, const int* starts, int nranks, int rank, int depth,
                       int depth_z, int r, bool viscous, int ndim, StripPlan* out);
int pow_tables_init();  // tables of the FP64 power on the current device, once per device; nonzero on a CUDA error

}  // namespace cfs
