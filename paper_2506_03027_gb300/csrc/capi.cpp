// capi.cpp -- the C ABI of libcfs (declared in include/cfs.h): context, decomposition,
// device memory, schedule and the per-step launch sequence of arXiv 2506.03027's method.
#include "cfs.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "cfs_internal.h"

using cfs::Geometry;
using cfs::Physics;
using cfs::StepSched;
using cfs::SubDev;

struct Block {
  int nx = 0, ny = 0, nz = 0;
  double h[3] = {1, 1, 1};
  int P[3] = {1, 1, 1};
  long long N = 0;        // points
  long long base = 0;     // offset of its state in a state array (doubles): 5 x points before it
  int sid0 = 0;           // index of its first sub-domain
  int* d_owner[3] = {nullptr, nullptr, nullptr};
  int* d_axis_off[3] = {nullptr, nullptr, nullptr};
  int* d_axis_len[3] = {nullptr, nullptr, nullptr};
  // curvilinear grid (cfs_set_block_grid): x, y of every (i, j), and the periodic coordinate jumps
  std::vector<double> xy;
  double shift[4] = {0, 0, 0, 0};
  long long mbase = -1;   // offset of its metric plane in d_metric
  cfs::FaceSpec face[6];  // periodic unless connected (cfs_connect) or bounded (cfs_set_bc)
  long long ebase = -1;   // offset of its gather map in d_emap (blocks with a non-periodic face)
};

struct cfs_ctx {
  cfs_params p{};
  std::vector<Block> blocks;
  cudaStream_t stream = nullptr;
  cfs_alloc_fn alloc = nullptr;
  cfs_free_fn freef = nullptr;
  void* user = nullptr;
  std::vector<void*> owned;

  bool finalized = false;

  int s = 0, C = 0, r = 0, G = 0, Gz = 0, ndim = 0;
  int max_delay = 0, R = 0;
  long long n = 0;
  double dt = 0.0;
  bool dt_set = false;
  double A[5] = {0}, B[5] = {0};

  int algo = 0, at = 1, L = 1;
  long long sched_steps = 0;
  int8_t* d_sched = nullptr;

  double* ring = nullptr;
  double* buf[2] = {nullptr, nullptr};
  double* Q = nullptr;
  void* Wp = nullptr;
  void* Phi = nullptr;
  double* d_W = nullptr;
  double* d_Wf = nullptr;
  float* d_W32 = nullptr;   // pairs of W for level-difference sums, then pairs of W - W^(0)
  float* d_W32d = nullptr;
  SubDev* d_subs = nullptr;
  std::vector<SubDev> subs;
  int max_pad = 0, max_own = 0, max_flux = 0;
  double* d_thomas = nullptr;
  float* d_thomas32 = nullptr;
  int Lmax = 0;
  double filt_h[6] = {0};
  double* d_partial = nullptr;
  double* d_out = nullptr;
  int diag_blocks = 0;

  // compact list of the halo points of every sub-domain: (sub-domain, padded index)
  int* d_halo = nullptr;
  long long nhalo = 0;

  // learned halo predictor
  bool learned = false;
  float* d_mlp = nullptr;
  double* LH = nullptr;
  float* d_mlpx = nullptr;   // the network's feature tiles: [ceil(ncol / MLP_TILE)][MLP_TILE x MLP_K1] FP32
  double* d_mlpa = nullptr;  // their 3-level extrapolations: [ceil(ncol / MLP_TILE)][MLP_TILE x MLP_NOUT] FP64
  int* d_cols = nullptr;
  long long ncol = 0;
  cfs::MlpScales mlp_scales{};

  // fused FP32-intermediate stage (3-D Navier-Stokes, CD4)
  bool fused = false;
  int fblock_n = 0;     // FP32 form, asynchronous steps: sub-domain filter for cubic sub-domains of this size
  float* d_fbhalo = nullptr;  // its halos: [nsub * 5][3][10][fblock_n^2] FP32 deviations
  int threads = 256;   // threads per CTA of the FP64 / 3-kernel stage kernels
  int fused_zc = 32;
  int fused_fy = 16;
  int fused_grid = 0;
  bool fused_curv = false;  // the fused stage runs curvilinear blocks (metric window in shared memory)
  double* d_metric = nullptr;  // metric planes of the curvilinear blocks
  int* d_emap = nullptr;       // gather maps of the blocks with non-periodic faces
  cfs::GatherEntry* d_gent = nullptr;
  bool all_periodic = true;
  double volume = 0.0;         // total cell volume (diagnostics averages)
  int nwork = 0;
  int* d_work = nullptr;
  float* Wh = nullptr;

  Geometry geo{};
  Physics phys{};

  std::string err;
  bool sticky = false;
  long long launches = 0;

  // CUDA graph of one step (device-resident step counter)
  long long* d_n = nullptr;
  bool graph_on = false;
  bool graph_dirty = true;
  cudaGraphExec_t gexec = nullptr;
  long long graph_launches = 0;  // kernel launches captured in one step

  // partitioned context (cfs_set_partition): this process computes sub-domains
  // [part_starts[part_rank], part_starts[part_rank + 1]); boundary strips travel through the
  // exchange callback
  int part_n = 1, part_rank = 0;
  std::vector<int> part_starts;
  cfs_exchange_fn xfn = nullptr;
  void* xuser = nullptr;
  std::vector<long long> x_send_cnt, x_recv_cnt;  // per peer, in doubles (5 x points)
  long long x_nsend = 0, x_nrecv = 0;             // points
  long long* d_x_send = nullptr;
  long long* d_x_recv = nullptr;
  int* d_x_send_n = nullptr;
  int* d_x_recv_n = nullptr;
  double* d_x_sbuf = nullptr;
  double* d_x_rbuf = nullptr;
  long long exchanges = 0;                        // callbacks made by the last cfs_step

  // device status word: bit 0 set by a bounded device wait that gave up
  int* d_status = nullptr;

  // compact scheme: the flux divergence [5][N] and the Thomas factors of its line systems
  double* Rbuf = nullptr;
  double* d_cthomas = nullptr;

  // per-kernel event timing
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<std::pair<int, size_t>> ev_pairs;  // (kind, index of the begin event)
  double t_ms[CFS_NKINDS] = {0};
  long long t_cnt[CFS_NKINDS] = {0};
  cfs::Timer timer{};
};

static void timer_rec(void* self, int kind, int begin) {
  cfs_ctx* c = (cfs_ctx*)self;
  if (c->ev_used == c->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    c->ev_pool.push_back(e);
  }
  const size_t idx = c->ev_used++;
  cudaEventRecord(c->ev_pool[idx], c->stream);
  if (begin) c->ev_pairs.push_back({kind, idx});
}

// Fold recorded event pairs into the per-kind totals (synchronises the stream).
static void timer_flush(cfs_ctx* c) {
  if (c->ev_pairs.empty()) { c->ev_used = 0; return; }
  cudaStreamSynchronize(c->stream);
  for (auto& pr : c->ev_pairs) {
    float ms = 0.f;
    if (pr.second + 1 < c->ev_used && cudaEventElapsedTime(&ms, c->ev_pool[pr.second], c->ev_pool[pr.second + 1]) == cudaSuccess) {
      c->t_ms[pr.first] += ms;
      c->t_cnt[pr.first] += 1;
    }
  }
  c->ev_pairs.clear();
  c->ev_used = 0;
}

static const char* kNoCtx = "null context";

static cfs_status fail(cfs_ctx* c, cfs_status st, const std::string& msg) {
  if (c) c->err = msg;
  return st;
}

static cfs_status cuda_fail(cfs_ctx* c, cudaError_t e, const char* where) {
  c->sticky = true;
  c->err = std::string(where) + ": " + cudaGetErrorString(e);
  return CFS_ECUDA;
}

#define CUDA_TRY(c, expr, where)                  \
  do {                                            \
    cudaError_t e_ = (expr);                      \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, where); \
  } while (0)

static void* default_alloc(size_t bytes, void*) {
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
  return p;
}
static void default_free(void* p, void*) { cudaFree(p); }

static void* dev_alloc(cfs_ctx* c, size_t bytes) {
  if (bytes == 0) bytes = 256;
  void* p = c->alloc(bytes, c->user);
  if (p) c->owned.push_back(p);
  return p;
}

static void dev_free(cfs_ctx* c, void* p) {
  if (!p) return;
  for (size_t i = 0; i < c->owned.size(); ++i)
    if (c->owned[i] == p) {
      c->owned.erase(c->owned.begin() + (long)i);
      c->freef(p, c->user);
      return;
    }
}

static void split_axis(int n, int p, int idx, int* off, int* len) {
  int base = n / p, rem = n % p;
  *len = base + (idx < rem ? 1 : 0);
  *off = idx * base + (idx < rem ? idx : rem);
}

extern "C" {

cfs_status cfs_create(const cfs_params* p, void* cuda_stream, cfs_ctx** out) {
  if (!p || !out) return CFS_EINVAL;
  *out = nullptr;
  if (p->order != 2 && p->order != 4) return CFS_EINVAL;
  if (p->precision != 0 && p->precision != 1) return CFS_EINVAL;
  if (p->filter && !(std::fabs(p->alpha_f) < 0.5)) return CFS_EINVAL;
  if (!(p->gamma > 1.0) || !(p->mach > 0.0) || (p->viscous && (!(p->re > 0.0) || !(p->pr > 0.0)))) return CFS_EINVAL;
  if (p->compact != 0 && (p->compact != 1 || p->viscous || p->order != 4 || p->precision != 0)) return CFS_EINVAL;
  cfs_ctx* c = new cfs_ctx();
  c->p = *p;
  c->stream = (cudaStream_t)cuda_stream;
  c->alloc = default_alloc;
  c->freef = default_free;
  c->s = cfs::lserk_coeffs(p->order, c->A, c->B);
  c->C = p->order == 4 ? 5 : 3;
  c->r = p->order == 4 ? 2 : 1;
  c->G = p->compact ? 4 : (p->viscous ? 2 * c->r : c->r);
  *out = c;
  return CFS_OK;
}

cfs_status cfs_set_allocator(cfs_ctx* c, cfs_alloc_fn alloc, cfs_free_fn free_fn, void* user) {
  if (!c) return CFS_EINVAL;
  if (c->finalized) return fail(c, CFS_ESTATE, "allocator must be set before cfs_finalize");
  if (!alloc || !free_fn) return fail(c, CFS_EINVAL, "allocator and free function required");
  c->alloc = alloc;
  c->freef = free_fn;
  c->user = user;
  return CFS_OK;
}

cfs_status cfs_add_block(cfs_ctx* c, int ni, int nj, int nk, const double* spacing, int* block_id) {
  if (!c) return CFS_EINVAL;
  if (c->finalized) return fail(c, CFS_ESTATE, "blocks must be added before cfs_finalize");
  if (ni < 1 || nj < 1 || nk < 1 || !spacing) return fail(c, CFS_EINVAL, "bad block size");
  for (int a = 0; a < 3; ++a)
    if (!(spacing[a] > 0.0)) return fail(c, CFS_EINVAL, "spacing must be positive");
  if ((long long)ni * nj * nk > (1LL << 31)) return fail(c, CFS_EINVAL, "block too large");
  const int ndim = nk > 1 ? 3 : 2;
  if (!c->blocks.empty() && ndim != c->ndim) return fail(c, CFS_EINVAL, "all blocks must be 2-D or all 3-D");
  if (c->blocks.size() >= 4096) return fail(c, CFS_EINVAL, "too many blocks");
  Block b;
  b.nx = ni; b.ny = nj; b.nz = nk;
  for (int a = 0; a < 3; ++a) b.h[a] = spacing[a];
  b.N = (long long)ni * nj * nk;
  c->blocks.push_back(b);
  c->ndim = ndim;
  c->Gz = nk > 1 ? c->G : 0;
  if (block_id) *block_id = (int)c->blocks.size() - 1;
  return CFS_OK;
}

cfs_status cfs_set_block_grid(cfs_ctx* c, int block, const double* xy, const double* shift) {
  if (!c) return CFS_EINVAL;
  if (c->finalized) return fail(c, CFS_ESTATE, "the grid must be set before cfs_finalize");
  if (block < 0 || block >= (int)c->blocks.size()) return fail(c, CFS_EINVAL, "unknown block");
  if (!xy || !shift) return fail(c, CFS_EINVAL, "null grid");
  Block& b = c->blocks[block];
  const size_t n2 = (size_t)b.nx * b.ny;
  for (size_t q = 0; q < 2 * n2; ++q)
    if (!std::isfinite(xy[q])) return fail(c, CFS_EINVAL, "non-finite grid coordinate");
  for (int k = 0; k < 4; ++k)
    if (!std::isfinite(shift[k])) return fail(c, CFS_EINVAL, "non-finite grid shift");
  b.xy.assign(xy, xy + 2 * n2);
  for (int k = 0; k < 4; ++k) b.shift[k] = shift[k];
  return CFS_OK;
}

cfs_status cfs_split_block(cfs_ctx* c, int block, int pi, int pj, int pk) {
  if (!c) return CFS_EINVAL;
  if (c->finalized) return fail(c, CFS_ESTATE, "split before cfs_finalize");
  if (block < 0 || block >= (int)c->blocks.size()) return fail(c, CFS_EINVAL, "unknown block");
  Block& b = c->blocks[block];
  if (pi < 1 || pj < 1 || pk < 1 || pi > b.nx || pj > b.ny || pk > b.nz) return fail(c, CFS_EINVAL, "bad split");
  b.P[0] = pi; b.P[1] = pj; b.P[2] = pk;
  return CFS_OK;
}

cfs_status cfs_connect(cfs_ctx* c, int blockA, int faceA, int blockB, int faceB, int orientation) {
  if (!c) return CFS_EINVAL;
  if (c->finalized) return fail(c, CFS_ESTATE, "connect before cfs_finalize");
  const int nb = (int)c->blocks.size();
  if (blockA < 0 || blockA >= nb || blockB < 0 || blockB >= nb) return fail(c, CFS_EINVAL, "unknown block");
  if (faceA < 0 || faceA > 5 || faceB < 0 || faceB > 5) return fail(c, CFS_EINVAL, "face must be 0..5");
  if (orientation != 0 && orientation != 1) return fail(c, CFS_EINVAL, "orientation must be 0 or 1");
  if (blockA == blockB && faceB == (faceA ^ 1) && orientation == 0) {  // periodic self-connection
    c->blocks[blockA].face[faceA] = cfs::FaceSpec{};
    c->blocks[blockA].face[faceB] = cfs::FaceSpec{};
    return CFS_OK;
  }
  if (faceA > 3 || faceB > 3) return fail(c, CFS_EINVAL, "interfaces join x or y faces (z is periodic)");
  if (blockA == blockB && faceA == faceB) return fail(c, CFS_EINVAL, "a face cannot join itself");
  cfs::FaceSpec fa, fb;
  fa.type = fb.type = cfs::FACE_INTERFACE;
  fa.nb = blockB; fa.nf = faceB; fa.rev = orientation;
  fb.nb = blockA; fb.nf = faceA; fb.rev = orientation;
  c->blocks[blockA].face[faceA] = fa;
  c->blocks[blockB].face[faceB] = fb;
  return CFS_OK;
}

cfs_status cfs_set_face_shift(cfs_ctx* c, int block, int face, const double* shift) {
  if (!c || !shift) return CFS_EINVAL;
  if (c->finalized) return fail(c, CFS_ESTATE, "face shift before cfs_finalize");
  if (block < 0 || block >= (int)c->blocks.size() || face < 0 || face > 3) return fail(c, CFS_EINVAL, "unknown block or face");
  cfs::FaceSpec& f = c->blocks[block].face[face];
  if (f.type != cfs::FACE_INTERFACE) return fail(c, CFS_EINVAL, "the face is not an interface");
  if (!std::isfinite(shift[0]) || !std::isfinite(shift[1])) return fail(c, CFS_EINVAL, "non-finite shift");
  f.shift[0] = shift[0];
  f.shift[1] = shift[1];
  return CFS_OK;
}

// The blocks' faces and grids as the host topology code sees them (validated); sid0 and base as
// cfs_finalize assigns them.
static const char* host_topology(cfs_ctx* c, std::vector<cfs::TopoBlock>& topo) {
  topo.assign(c->blocks.size(), cfs::TopoBlock{});
  int sid0 = 0;
  long long base = 0;
  for (size_t bi = 0; bi < c->blocks.size(); ++bi) {
    const Block& b = c->blocks[bi];
    cfs::TopoBlock& t = topo[bi];
    t.n[0] = b.nx; t.n[1] = b.ny; t.n[2] = b.nz;
    for (int a = 0; a < 3; ++a) t.P[a] = b.P[a];
    t.sid0 = sid0;
    t.base = base;
    t.N = b.N;
    t.xy = b.xy.empty() ? nullptr : b.xy.data();
    for (int q = 0; q < 4; ++q) t.shift[q] = b.shift[q];
    for (int f = 0; f < 6; ++f) t.face[f] = b.face[f];
    sid0 += b.P[0] * b.P[1] * b.P[2];
    base += 5 * b.N;
  }
  return cfs::topo_check(topo.data(), (int)topo.size());
}

cfs_status cfs_metric_terms(cfs_ctx* c, int block, int i, int j, double* out) {
  if (!c || !out) return CFS_EINVAL;
  if (block < 0 || block >= (int)c->blocks.size()) return fail(c, CFS_EINVAL, "unknown block");
  const Block& b = c->blocks[block];
  if (b.xy.empty()) return fail(c, CFS_EINVAL, "the block is Cartesian");
  if (i < -c->G || i >= b.nx + c->G || j < -c->G || j >= b.ny + c->G)
    return fail(c, CFS_EINVAL, "point farther than the halo depth from the block");
  std::vector<cfs::TopoBlock> topo;
  if (const char* why = host_topology(c, topo)) return fail(c, CFS_EINVAL, why);
  const int mx = b.nx + 2 * c->G, my = b.ny + 2 * c->G;
  std::vector<double> M((size_t)NMETRIC * mx * my);
  if (!cfs::metric_plane(topo.data(), (int)topo.size(), block, c->G, c->r, c->p.order, b.h[2], b.nz > 1 ? 3 : 2, M.data()))
    return fail(c, CFS_EINVAL, "curvilinear grid with a non-positive cell volume, or not continued across a face");
  const size_t pl = (size_t)mx * my, at = (size_t)(i + c->G) + (size_t)mx * (j + c->G);
  for (int q = 0; q < NMETRIC; ++q) out[q] = M[q * pl + at];
  return CFS_OK;
}

cfs_status cfs_halo_sources(cfs_ctx* c, int block, int i, int j, int k, double* out) {
  if (!c || !out) return CFS_EINVAL;
  if (block < 0 || block >= (int)c->blocks.size()) return fail(c, CFS_EINVAL, "unknown block");
  std::vector<cfs::TopoBlock> topo;
  if (const char* why = host_topology(c, topo)) return fail(c, CFS_EINVAL, why);
  const Block& b = c->blocks[block];
  const int G = c->p.filter ? std::max(c->G, 5) : c->G;
  if (i < -G || i >= b.nx + G || j < -G || j >= b.ny + G || k < -G || k >= b.nz + G)
    return fail(c, CFS_EINVAL, "point farther than the halo depth from the block");
  if (cfs::halo_sources(topo.data(), (int)topo.size(), block, i, j, k, out) < 0)
    return fail(c, CFS_EINVAL, "the point does not resolve");
  return CFS_OK;
}

cfs_status cfs_set_bc(cfs_ctx* c, int block, int face, int type, const double* data) {
  if (!c) return CFS_EINVAL;
  if (c->finalized) return fail(c, CFS_ESTATE, "boundary conditions before cfs_finalize");
  if (block < 0 || block >= (int)c->blocks.size()) return fail(c, CFS_EINVAL, "unknown block");
  if (face < 0 || face > 3) return fail(c, CFS_EINVAL, "boundaries lie on x or y faces (z is periodic)");
  cfs::FaceSpec f;
  switch (type) {
    case CFS_BC_PERIODIC:
      c->blocks[block].face[face] = f;
      c->blocks[block].face[face ^ 1] = f;
      return CFS_OK;
    case CFS_BC_WALL: f.type = cfs::FACE_WALL; break;
    case CFS_BC_OUTFLOW: f.type = cfs::FACE_OUTFLOW; break;
    case CFS_BC_FARFIELD:
      if (!data) return fail(c, CFS_EINVAL, "far field needs its conserved state");
      for (int v = 0; v < 5; ++v) {
        if (!std::isfinite(data[v])) return fail(c, CFS_EINVAL, "non-finite far-field state");
        f.state[v] = data[v];
      }
      if (!(data[0] > 0.0)) return fail(c, CFS_EINVAL, "far-field density must be positive");
      f.type = cfs::FACE_FARFIELD;
      break;
    default:
      return fail(c, CFS_EINVAL, "unknown boundary type");
  }
  c->blocks[block].face[face] = f;
  return CFS_OK;
}

cfs_status cfs_finalize(cfs_ctx* c, int max_delay) {
  if (!c) return CFS_EINVAL;
  if (c->finalized) return fail(c, CFS_ESTATE, "already finalized");
  if (c->blocks.empty()) return fail(c, CFS_ESTATE, "no block");
  if (max_delay < 0 || max_delay > CFS_MAX_DELAY) return fail(c, CFS_EINVAL, "max_delay out of range");
  const int need = c->p.filter ? (c->G > 5 ? c->G : 5) : c->G;
  // sub-domain table: blocks in order, x fastest within a block
  int nsub = 0;
  long long Ntot = 0, mtot = 0;
  for (Block& b : c->blocks) {
    b.sid0 = nsub;
    b.base = 5 * Ntot;
    b.mbase = b.xy.empty() ? -1 : mtot;
    if (!b.xy.empty()) mtot += (long long)NMETRIC * (b.nx + 2 * c->G) * (b.ny + 2 * c->G);
    nsub += b.P[0] * b.P[1] * b.P[2];
    Ntot += b.N;
  }
  // block topology: faces, gather maps of the blocks with a non-periodic face
  std::vector<cfs::TopoBlock> topo;
  if (const char* why = host_topology(c, topo)) return fail(c, CFS_EINVAL, why);
  c->all_periodic = true;
  for (const cfs::TopoBlock& t : topo) c->all_periodic = c->all_periodic && cfs::topo_periodic(t);
  c->subs.resize(nsub);
  long long pbase = 0;
  c->max_pad = c->max_own = c->max_flux = 0;
  const int fs = c->p.compact ? 4 : c->r;  // flux strips beyond each face
  const int rz = c->ndim == 3 ? fs : 0;
  const double a_cd = c->p.order == 4 ? 4.0 / 3.0 : 1.0, b_cd = c->p.order == 4 ? -1.0 / 3.0 : 0.0;
  for (const Block& b : c->blocks)
    for (int iz = 0; iz < b.P[2]; ++iz)
      for (int iy = 0; iy < b.P[1]; ++iy)
        for (int ix = 0; ix < b.P[0]; ++ix) {
          SubDev d{};
          split_axis(b.nx, b.P[0], ix, &d.ox, &d.sx);
          split_axis(b.ny, b.P[1], iy, &d.oy, &d.sy);
          split_axis(b.nz, b.P[2], iz, &d.oz, &d.sz);
          if (d.sx < need || d.sy < need || (c->ndim == 3 && d.sz < need))
            return fail(c, CFS_EINVAL, "sub-domain smaller than the halo it needs");
          d.ex = d.sx + 2 * c->G;
          d.ey = d.sy + 2 * c->G;
          d.ez = d.sz + 2 * c->Gz;
          d.ix = ix; d.iy = iy; d.iz = iz;
          d.pbase = pbase;
          d.bnx = b.nx; d.bny = b.ny; d.bnz = b.nz;
          d.bN = b.N;
          d.bbase = b.base;
          d.mbase = b.mbase;
          d.mx = b.nx + 2 * c->G;
          d.mpl = (long long)(b.nx + 2 * c->G) * (b.ny + 2 * c->G);
          d.phys = d.wall = 0;
          {
            const int lo[3] = {d.ox, d.oy, d.oz}, hi[3] = {d.ox + d.sx, d.oy + d.sy, d.oz + d.sz};
            const int n3[3] = {b.nx, b.ny, b.nz};
            for (int a = 0; a < 3; ++a)
              for (int side = 0; side < 2; ++side) {
                const int f = 2 * a + side;
                const bool on = side == 0 ? lo[a] == 0 : hi[a] == n3[a];
                if (on && b.face[f].type >= cfs::FACE_WALL) d.phys |= 1 << f;
                if (on && b.face[f].type == cfs::FACE_WALL) d.wall |= 1 << f;
              }
          }
          d.ebase = -1;
          d.own = 1;
          d.gmx = b.nx + 2 * need;
          d.gmy = b.ny + 2 * need;
          for (int a = 0; a < 3; ++a) {  // CD coefficients of Eq. 2 (alpha = 0) for the block's spacing
            const double h = b.mbase >= 0 ? 1.0 : b.h[a];  // curvilinear: index space
            d.c1[a] = (a_cd / 2.0) / h;
            d.c2[a] = (b_cd / 4.0) / h;
          }
          const long long npad = (long long)d.ex * d.ey * d.ez;
          pbase += npad;
          const long long nown = (long long)d.sx * d.sy * d.sz;
          const long long nfl = (long long)(d.sx + 2 * fs) * (d.sy + 2 * fs) * (d.sz + 2 * rz);
          if (npad > (1LL << 30)) return fail(c, CFS_EINVAL, "sub-domain too large");
          c->max_pad = (int)std::max<long long>(c->max_pad, npad);
          c->max_own = (int)std::max<long long>(c->max_own, nown);
          c->max_flux = (int)std::max<long long>(c->max_flux, nfl);
          c->subs[b.sid0 + ix + b.P[0] * (iy + b.P[1] * iz)] = d;
        }
  // partitioned context: validate, mark the sub-domains another process computes
  const bool parted = c->part_n > 1;
  cfs::StripPlan plan;
  if (parted) {
    if (c->p.precision != 0 || c->learned) return fail(c, CFS_EINVAL, "a partitioned context runs the FP64 path only");
    if ((int)c->part_starts.size() != c->part_n + 1 || c->part_starts[c->part_n] != nsub)
      return fail(c, CFS_EINVAL, "the partition does not cover the sub-domains");
    for (int sid = 0; sid < nsub; ++sid)
      c->subs[sid].own = (sid >= c->part_starts[c->part_rank] && sid < c->part_starts[c->part_rank + 1]) ? 1 : 0;
    const int depth = need, depth_z = c->ndim == 3 ? need : 0;
    if (const char* why = cfs::strip_plan(topo.data(), (int)topo.size(), nsub, c->part_starts.data(), c->part_n,
                                          c->part_rank, depth, depth_z, c->r, c->p.viscous != 0, c->ndim, &plan))
      return fail(c, CFS_EINVAL, why);
  }
  c->max_delay = max_delay;
  c->R = max_delay + c->C + 1;
  const long long N = Ntot;
  const Block& b0 = c->blocks[0];
  const size_t tsz = c->p.precision == 1 ? sizeof(float) : sizeof(double);
  // geometry / physics
  Geometry& g = c->geo;
  g.nx = b0.nx; g.ny = b0.ny; g.nz = b0.nz; g.N = N; g.nsub = nsub;
  g.G = c->G; g.Gz = c->Gz; g.r = c->r; g.ndim = c->ndim; g.viscous = c->p.viscous; g.Ptot = pbase;
  g.fs = fs;
  Physics& ph = c->phys;
  ph.gamma = c->p.gamma; ph.gm1 = c->p.gamma - 1.0; ph.gM2 = c->p.gamma * c->p.mach * c->p.mach;
  ph.ire = c->p.viscous ? 1.0 / c->p.re : 0.0;
  ph.kappa = c->p.viscous ? 1.0 / ((c->p.gamma - 1.0) * c->p.pr * c->p.mach * c->p.mach) : 0.0;
  ph.visc_law = c->p.visc_law; ph.visc_exp = c->p.visc_exp;
  ph.kgM2 = ph.kappa * ph.gM2;
  ph.ivT = (c->p.viscous && c->p.visc_law == 1) ? ph.ire * std::pow(ph.kappa, -c->p.visc_exp) : ph.ire;
  ph.p_ref = 1.0 / ph.gM2;
  ph.E_ref = ph.p_ref / ph.gm1;
  ph.H_ref = ph.E_ref + ph.p_ref;
  // CD coefficients of Eq. 2 with alpha = 0 (CD4 a = 4/3, b = -1/3; CD2 a = 1, b = 0) of the
  // first block; each sub-domain carries those of its own block
  for (int a = 0; a < 3; ++a) {
    ph.c1[a] = (a_cd / 2.0) / b0.h[a];
    ph.c2[a] = (b_cd / 4.0) / b0.h[a];
  }
  // tables of the FP64 power (power-law viscosity)
  if (c->p.viscous && c->p.visc_law == 1) {
    const int rc = cfs::pow_tables_init();
    if (rc != 0) return cuda_fail(c, (cudaError_t)rc, "power tables");
  }
  // device memory
  c->ring = (double*)dev_alloc(c, sizeof(double) * 5 * N * c->R);
  c->buf[0] = (double*)dev_alloc(c, sizeof(double) * 5 * N);
  c->buf[1] = (double*)dev_alloc(c, sizeof(double) * 5 * N);
  c->Q = (double*)dev_alloc(c, sizeof(double) * 5 * N);
  // metric fields of the curvilinear blocks, and the total volume for the diagnostics
  bool curv = false;
  c->volume = 0.0;
  for (const Block& b : c->blocks) {
    curv = curv || b.mbase >= 0;
    if (b.mbase < 0) c->volume += (double)b.N * b.h[0] * b.h[1] * (c->ndim == 3 ? b.h[2] : 1.0);
  }
  if (curv) {
    c->d_metric = (double*)dev_alloc(c, sizeof(double) * mtot);
    if (!c->d_metric) return fail(c, CFS_ENOMEM, "device allocation failed");
    std::vector<double> M;
    for (size_t bi = 0; bi < c->blocks.size(); ++bi) {
      const Block& b = c->blocks[bi];
      if (b.mbase < 0) continue;
      const int mx = b.nx + 2 * c->G;
      const long long pl = (long long)mx * (b.ny + 2 * c->G);
      M.assign((size_t)NMETRIC * pl, 0.0);
      if (!cfs::metric_plane(topo.data(), (int)topo.size(), (int)bi, c->G, c->r, c->p.order, b.h[2], c->ndim, M.data()))
        return fail(c, CFS_EINVAL, "curvilinear grid with a non-positive cell volume, or not continued across a face");
      double vb = 0.0;
      for (int j = 0; j < b.ny; ++j)
        for (int i = 0; i < b.nx; ++i) vb += M[5 * pl + (i + c->G) + (long long)mx * (j + c->G)];
      c->volume += vb * b.nz;
      CUDA_TRY(c, cudaMemcpy(c->d_metric + b.mbase, M.data(), sizeof(double) * M.size(), cudaMemcpyHostToDevice),
               "upload metrics");
    }
  }
  g.metric = c->d_metric;
  // gather maps: every point of a non-periodic block's (x, y) range extended by `need` (faces to
  // that depth, corners to r x r), all z; entries for the points outside the block
  g.GE = need;
  g.emap = nullptr;
  g.gent = nullptr;
  bool simple_own = true;  // every entry with a source reached without crossing is one unit copy of it
  if (!c->all_periodic) {
    std::vector<int> emap;
    std::vector<cfs::GatherEntry> ent;
    for (size_t bi = 0; bi < c->blocks.size(); ++bi) {
      Block& b = c->blocks[bi];
      if (cfs::topo_periodic(topo[bi])) continue;
      b.ebase = (long long)emap.size();
      const int gx = b.nx + 2 * need, gy = b.ny + 2 * need;
      for (int k = 0; k < b.nz; ++k)
        for (int j = -need; j < b.ny + need; ++j)
          for (int i = -need; i < b.nx + need; ++i) {
            const int di = i < 0 ? -i : (i >= b.nx ? i - b.nx + 1 : 0);
            const int dj = j < 0 ? -j : (j >= b.ny ? j - b.ny + 1 : 0);
            if ((di == 0 && dj == 0) || (di && dj && (di > c->r || dj > c->r))) {
              emap.push_back(-1);
              continue;
            }
            cfs::GatherEntry e;
            if (!cfs::gather_entry(topo.data(), (int)topo.size(), (int)bi, i, j, k, &e))
              return fail(c, CFS_EINVAL, "a halo point beyond a block face does not resolve (more than 4 sources, "
                                         "or a face sequence that does not end inside a block)");
            if (ent.size() >= (size_t)INT32_MAX) return fail(c, CFS_EINVAL, "too many gather entries");
            emap.push_back((int)ent.size());
            ent.push_back(e);
            bool uncrossed = false;
            for (int q = 0; q < e.nt; ++q) uncrossed = uncrossed || !(e.flags[q] & 2);
            if (uncrossed && !(e.nt == 1 && e.w[0] == 1.0 && e.cst[0] == 0.0 && e.cst[1] == 0.0 && e.cst[2] == 0.0 &&
                               e.cst[3] == 0.0 && e.cst[4] == 0.0))
              simple_own = false;
          }
      (void)gx; (void)gy;
    }
    c->d_emap = (int*)dev_alloc(c, sizeof(int) * emap.size());
    c->d_gent = (cfs::GatherEntry*)dev_alloc(c, sizeof(cfs::GatherEntry) * ent.size());
    if (!c->d_emap || !c->d_gent) return fail(c, CFS_ENOMEM, "device allocation failed");
    CUDA_TRY(c, cudaMemcpy(c->d_emap, emap.data(), sizeof(int) * emap.size(), cudaMemcpyHostToDevice), "upload gather map");
    CUDA_TRY(c, cudaMemcpy(c->d_gent, ent.data(), sizeof(cfs::GatherEntry) * ent.size(), cudaMemcpyHostToDevice),
             "upload gather entries");
    g.emap = c->d_emap;
    g.gent = c->d_gent;
    for (const Block& b : c->blocks)
      for (int q = 0; q < b.P[0] * b.P[1] * b.P[2]; ++q) c->subs[b.sid0 + q].ebase = b.ebase;
  }
  // the fused FP32 stage: 3-D Navier-Stokes CD4; on connected grids its halo gather takes wall
  // mirrors / outflow copies as one unit copy of an own point of the same plane
  c->fused = c->p.precision == 1 && c->ndim == 3 && c->p.viscous && c->p.order == 4 && simple_own;
  c->fused_curv = curv;
  c->fblock_n = 0;
  if (c->p.precision == 1 && c->p.filter && c->ndim == 3 && !curv && c->all_periodic && nsub > 0) {
    const int n0 = c->subs[0].sx;
    bool cubic = cfs::filter_block_supported(n0);
    for (const SubDev& d : c->subs) cubic = cubic && d.sx == n0 && d.sy == n0 && d.sz == n0;
    if (cubic) {
      c->fblock_n = n0;
      c->d_fbhalo = (float*)dev_alloc(c, sizeof(float) * (size_t)nsub * 15 * 10 * n0 * n0);
      if (!c->d_fbhalo) return fail(c, CFS_ENOMEM, "device allocation failed");
    }
  }
  if (c->fused) {
    // tiles of 32 x fy columns per sub-domain, marching z; one CTA per tile (persistent grid)
    std::vector<int> work;
    for (int sid = 0; sid < nsub; ++sid) {
      const SubDev& d = c->subs[sid];
      for (int z0 = 0; z0 < d.sz; z0 += c->fused_zc)
        for (int y0 = 0; y0 < d.sy; y0 += c->fused_fy)
          for (int x0 = 0; x0 < d.sx; x0 += 32) {
            const int z1 = std::min(d.sz, z0 + c->fused_zc);
            work.push_back(sid); work.push_back(x0); work.push_back(y0); work.push_back(z0 | (z1 << 16));
          }
    }
    c->nwork = (int)(work.size() / 4);
    c->d_work = (int*)dev_alloc(c, sizeof(int) * work.size());
    c->Wh = (float*)dev_alloc(c, sizeof(float) * 7 * c->s * (size_t)pbase);
    if (!c->d_work || !c->Wh) return fail(c, CFS_ENOMEM, "device allocation failed");
    CUDA_TRY(c, cudaMemcpy(c->d_work, work.data(), sizeof(int) * work.size(), cudaMemcpyHostToDevice), "upload work list");
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int per_sm = 0;
    if (cfs::fused_blocks_per_sm(c->fused_fy, curv ? 1 : 0, &per_sm) != 0 || per_sm < 1)
      return fail(c, CFS_ECUDA, "fused stage kernel does not fit on this device");
    c->fused_grid = std::max(1, std::min(c->nwork, per_sm * std::max(1, sms)));
  } else {
    c->Wp = dev_alloc(c, tsz * 7 * (size_t)pbase);
    c->Phi = dev_alloc(c, tsz * 15 * (size_t)pbase);
  }
  c->d_subs = (SubDev*)dev_alloc(c, sizeof(SubDev) * nsub);
  const int nW = (max_delay + 1) * c->s * c->C, nWf = (max_delay + 1) * c->C;
  c->d_W = (double*)dev_alloc(c, sizeof(double) * nW);
  c->d_Wf = (double*)dev_alloc(c, sizeof(double) * nWf);
  c->d_W32 = (float*)dev_alloc(c, sizeof(float) * 4 * nW);
  c->d_W32d = c->d_W32 ? c->d_W32 + 2 * (size_t)nW : nullptr;
  c->d_out = (double*)dev_alloc(c, sizeof(double) * 8);
  c->d_n = (long long*)dev_alloc(c, sizeof(long long));
  c->d_status = (int*)dev_alloc(c, sizeof(int));
  c->Lmax = 0;
  for (Block& b : c->blocks) {
    const int n3[3] = {b.nx, b.ny, b.nz};
    for (int a = 0; a < 3; ++a) {
      b.d_owner[a] = (int*)dev_alloc(c, sizeof(int) * n3[a]);
      b.d_axis_off[a] = (int*)dev_alloc(c, sizeof(int) * b.P[a]);
      b.d_axis_len[a] = (int*)dev_alloc(c, sizeof(int) * b.P[a]);
      c->Lmax = std::max(c->Lmax, (n3[a] + b.P[a] - 1) / b.P[a]);
    }
  }
  if (c->p.compact) {
    for (const Block& b : c->blocks)
      if (b.mbase >= 0) return fail(c, CFS_EINVAL, "the compact scheme runs on Cartesian blocks");
    if (!c->all_periodic) return fail(c, CFS_EINVAL, "the compact scheme needs blocks periodic on every face");
    if (c->Lmax > CFS_MAX_LINE) return fail(c, CFS_EINVAL, "the compact scheme's sub-domain lines are limited to 128 points");
    c->Rbuf = (double*)dev_alloc(c, sizeof(double) * 5 * (size_t)N);
    c->d_cthomas = (double*)dev_alloc(c, sizeof(double) * (size_t)(c->Lmax + 1) * 2 * c->Lmax);
    if (!c->Rbuf || !c->d_cthomas) return fail(c, CFS_ENOMEM, "device allocation failed");
    // Thomas factors of the compact system (unit diagonal, off-diagonals 1/3) per line length
    std::vector<double> ct((size_t)(c->Lmax + 1) * 2 * c->Lmax, 0.0);
    const double al = 1.0 / 3.0;
    for (int len = 1; len <= c->Lmax; ++len) {
      double* cp = ct.data() + (size_t)len * 2 * c->Lmax;
      double* im = cp + c->Lmax;
      double m = 1.0;
      cp[0] = al;
      im[0] = 1.0;
      for (int i = 1; i < len; ++i) {
        m = 1.0 - al * cp[i - 1];
        cp[i] = al / m;
        im[i] = 1.0 / m;
      }
    }
    CUDA_TRY(c, cudaMemcpy(c->d_cthomas, ct.data(), sizeof(double) * ct.size(), cudaMemcpyHostToDevice), "upload compact factors");
  }
  if (c->p.filter && cfs::filter_prepare(c->Lmax, c->p.precision) != 0)
    return fail(c, CFS_EINVAL, "filter: a sub-domain is too long along an axis for the shared-memory line tiles "
                               "(at most about 700 points)");
  c->diag_blocks = 2 * 152;
  c->d_partial = (double*)dev_alloc(c, sizeof(double) * DIAG_NQ * c->diag_blocks * c->blocks.size());
  c->d_thomas = (double*)dev_alloc(c, sizeof(double) * (size_t)(c->Lmax + 1) * 2 * c->Lmax);
  c->d_thomas32 = (float*)dev_alloc(c, sizeof(float) * (size_t)(c->Lmax + 1) * 2 * c->Lmax);
  for (void* q : c->owned)
    if (!q) return fail(c, CFS_ENOMEM, "device allocation failed");
  if (!c->d_n || !c->d_status || !c->ring || !c->buf[0] || !c->buf[1] || !c->Q || (!c->fused && (!c->Wp || !c->Phi)) || !c->d_subs || !c->d_W || !c->d_Wf || !c->d_W32 ||
      !c->d_partial || !c->d_out || !c->d_thomas || !c->d_thomas32)
    return fail(c, CFS_ENOMEM, "device allocation failed");
  for (const Block& b : c->blocks)
    for (int a = 0; a < 3; ++a)
      if (!b.d_owner[a] || !b.d_axis_off[a] || !b.d_axis_len[a]) return fail(c, CFS_ENOMEM, "device allocation failed");
  // halo list: faces to depth G, viscous edges to r x r (the points each sub-domain reads from
  // its neighbours)
  {
    std::vector<int> hl;
    for (int sid = 0; sid < nsub; ++sid) {
      const SubDev& d = c->subs[sid];
      if (!d.own) continue;  // computed by another process
      for (int k = 0; k < d.ez; ++k)
        for (int j = 0; j < d.ey; ++j)
          for (int i = 0; i < d.ex; ++i) {
            const int ci = i - c->G, cj = j - c->G, ck = k - c->Gz;
            const int dx = ci < 0 ? -ci : (ci >= d.sx ? ci - d.sx + 1 : 0);
            const int dy = cj < 0 ? -cj : (cj >= d.sy ? cj - d.sy + 1 : 0);
            const int dz = ck < 0 ? -ck : (ck >= d.sz ? ck - d.sz + 1 : 0);
            const int nout = (dx > 0) + (dy > 0) + (dz > 0);
            const bool need = nout == 1 || (nout == 2 && c->p.viscous && dx <= c->r && dy <= c->r && dz <= c->r);
            if (!need) continue;
            hl.push_back(sid);
            hl.push_back(i + d.ex * (j + d.ey * k));
          }
    }
    c->nhalo = (long long)(hl.size() / 2);
    if (c->nhalo > 0) {
      c->d_halo = (int*)dev_alloc(c, sizeof(int) * hl.size());
      if (!c->d_halo) return fail(c, CFS_ENOMEM, "device allocation failed");
      CUDA_TRY(c, cudaMemcpy(c->d_halo, hl.data(), sizeof(int) * hl.size(), cudaMemcpyHostToDevice), "upload halo list");
    }
  }
  // exchange plan of a partitioned context: state offsets and block sizes of the strips sent to /
  // received from every peer, and the packed buffers (5 values per point)
  if (parted) {
    c->x_nsend = (long long)plan.send.size();
    c->x_nrecv = (long long)plan.recv.size();
    c->x_send_cnt.assign(c->part_n, 0);
    c->x_recv_cnt.assign(c->part_n, 0);
    for (int q = 0; q < c->part_n; ++q) {
      c->x_send_cnt[q] = 5 * (plan.send_off[q + 1] - plan.send_off[q]);
      c->x_recv_cnt[q] = 5 * (plan.recv_off[q + 1] - plan.recv_off[q]);
    }
    c->d_x_send = (long long*)dev_alloc(c, sizeof(long long) * (c->x_nsend + 1));
    c->d_x_recv = (long long*)dev_alloc(c, sizeof(long long) * (c->x_nrecv + 1));
    c->d_x_send_n = (int*)dev_alloc(c, sizeof(int) * (c->x_nsend + 1));
    c->d_x_recv_n = (int*)dev_alloc(c, sizeof(int) * (c->x_nrecv + 1));
    c->d_x_sbuf = (double*)dev_alloc(c, sizeof(double) * 5 * (c->x_nsend + 1));
    c->d_x_rbuf = (double*)dev_alloc(c, sizeof(double) * 5 * (c->x_nrecv + 1));
    if (!c->d_x_send || !c->d_x_recv || !c->d_x_send_n || !c->d_x_recv_n || !c->d_x_sbuf || !c->d_x_rbuf)
      return fail(c, CFS_ENOMEM, "device allocation failed");
    if (c->x_nsend) {
      CUDA_TRY(c, cudaMemcpy(c->d_x_send, plan.send.data(), sizeof(long long) * c->x_nsend, cudaMemcpyHostToDevice), "upload plan");
      CUDA_TRY(c, cudaMemcpy(c->d_x_send_n, plan.send_bN.data(), sizeof(int) * c->x_nsend, cudaMemcpyHostToDevice), "upload plan");
    }
    if (c->x_nrecv) {
      CUDA_TRY(c, cudaMemcpy(c->d_x_recv, plan.recv.data(), sizeof(long long) * c->x_nrecv, cudaMemcpyHostToDevice), "upload plan");
      CUDA_TRY(c, cudaMemcpy(c->d_x_recv_n, plan.recv_bN.data(), sizeof(int) * c->x_nrecv, cudaMemcpyHostToDevice), "upload plan");
    }
  }
  // host tables
  std::vector<double> W(nW), Wf(nWf);
  if (cfs::at_weight_table(c->p.order, max_delay, W.data()) != nW ||
      cfs::filter_extrap_table(c->p.order, max_delay, Wf.data()) != nWf)
    return fail(c, CFS_EINVAL, "coefficient generation failed");
  // the AT weights for sums over the differences of the delayed levels from the newest one, as
  // pairs of floats (hi, lo = the rest of the FP64 value): per delay and stage S - 1 (S = sum_l W_l,
  // summed in a fixed order) and W_1 .. W_{C-1}; then the same for W^(m) - W^(0)
  std::vector<float> W32(4 * (size_t)nW);
  auto pair = [&](size_t i, double x) {
    W32[2 * i] = (float)x;
    W32[2 * i + 1] = (float)(x - (double)W32[2 * i]);
  };
  for (int tab = 0; tab < 2; ++tab)
    for (int km = 0; km < nW / c->C; ++km) {
      const double* w = W.data() + (size_t)km * c->C;
      const double* w0 = W.data() + (size_t)(km - km % c->s) * c->C;  // stage 0 of the same delay
      double x[CFS_MAX_LEVELS], sum = 0.0;
      for (int l = 0; l < c->C; ++l) {
        x[l] = tab ? w[l] - w0[l] : w[l];
        sum += x[l];
      }
      const size_t base = (size_t)tab * nW + (size_t)km * c->C;
      pair(base, tab ? sum : sum - 1.0);
      for (int l = 1; l < c->C; ++l) pair(base + l, x[l]);
    }
  double filt[6] = {1, 0, 0, 0, 0, 0};
  if (c->p.filter && !cfs::pade10_coeffs(c->p.alpha_f, filt)) return fail(c, CFS_EINVAL, "filter coefficients failed");
  c->filt_h[0] = filt[0];
  for (int m = 1; m < 6; ++m) c->filt_h[m] = 0.5 * filt[m];
  std::vector<double> th((size_t)(c->Lmax + 1) * 2 * c->Lmax, 0.0);
  const double al = c->p.alpha_f;
  for (int len = 1; len <= c->Lmax; ++len) {
    double* cp = th.data() + (size_t)len * 2 * c->Lmax;
    double* im = cp + c->Lmax;
    double m = 1.0;
    cp[0] = al / m;
    im[0] = 1.0 / m;
    for (int i = 1; i < len; ++i) {
      m = 1.0 - al * cp[i - 1];
      cp[i] = al / m;
      im[i] = 1.0 / m;
    }
  }
  cudaStream_t st = c->stream;
  CUDA_TRY(c, cudaMemcpyAsync(c->d_subs, c->subs.data(), sizeof(SubDev) * nsub, cudaMemcpyHostToDevice, st), "upload sub-domains");
  CUDA_TRY(c, cudaMemcpyAsync(c->d_W, W.data(), sizeof(double) * nW, cudaMemcpyHostToDevice, st), "upload weights");
  CUDA_TRY(c, cudaMemcpyAsync(c->d_Wf, Wf.data(), sizeof(double) * nWf, cudaMemcpyHostToDevice, st), "upload weights");
  CUDA_TRY(c, cudaMemcpyAsync(c->d_W32, W32.data(), sizeof(float) * W32.size(), cudaMemcpyHostToDevice, st), "upload weights");
  CUDA_TRY(c, cudaMemcpyAsync(c->d_thomas, th.data(), sizeof(double) * th.size(), cudaMemcpyHostToDevice, st), "upload filter");
  {
    const int rc = cfs::launch_round_table(c->d_thomas, c->d_thomas32, (long long)th.size(), st);
    if (rc != 0) return cuda_fail(c, (cudaError_t)rc, "filter table");
  }
  std::vector<std::vector<int>> keep;  // host tables stay alive until the stream is synchronised below
  for (Block& b : c->blocks) {
    const int n3[3] = {b.nx, b.ny, b.nz};
    for (int a = 0; a < 3; ++a) {
      std::vector<int> owner(n3[a]), aoff(b.P[a]), alen(b.P[a]);
      for (int i = 0; i < b.P[a]; ++i) {
        split_axis(n3[a], b.P[a], i, &aoff[i], &alen[i]);
        for (int t = 0; t < alen[i]; ++t) owner[aoff[i] + t] = i;
      }
      keep.push_back(owner); keep.push_back(aoff); keep.push_back(alen);
      const size_t k0 = keep.size() - 3;
      CUDA_TRY(c, cudaMemcpyAsync(b.d_owner[a], keep[k0].data(), sizeof(int) * n3[a], cudaMemcpyHostToDevice, st), "upload tables");
      CUDA_TRY(c, cudaMemcpyAsync(b.d_axis_off[a], keep[k0 + 1].data(), sizeof(int) * b.P[a], cudaMemcpyHostToDevice, st), "upload tables");
      CUDA_TRY(c, cudaMemcpyAsync(b.d_axis_len[a], keep[k0 + 2].data(), sizeof(int) * b.P[a], cudaMemcpyHostToDevice, st), "upload tables");
    }
  }
  CUDA_TRY(c, cudaMemsetAsync(c->ring, 0, sizeof(double) * 5 * N * c->R, st), "clear ring");
  CUDA_TRY(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), st), "clear status");
  // the host vectors above are pageable: make sure the copies have consumed them
  CUDA_TRY(c, cudaStreamSynchronize(st), "finalize");
  c->finalized = true;
  c->n = 0;
  return CFS_OK;
}

cfs_status cfs_set_schedule(cfs_ctx* c, int algo, int at, int L, long long nsteps, const int8_t* delays) {
  if (!c) return CFS_EINVAL;
  if (!c->finalized) return fail(c, CFS_ESTATE, "schedule after cfs_finalize");
  if (algo < 0 || algo > 2) return fail(c, CFS_EINVAL, "algo must be 0 (SA), 1 (CAA) or 2 (SAA)");
  if (algo == 1 && (L < 1 || L - 1 > c->max_delay)) return fail(c, CFS_EINVAL, "CAA needs 1 <= L <= max_delay + 1");
  if (algo == 2) {
    if (nsteps < 1 || !delays) return fail(c, CFS_EINVAL, "SAA needs a delay table");
    const long long cnt = nsteps * (long long)c->subs.size() * 6;
    for (long long i = 0; i < cnt; ++i)
      if (delays[i] < 0 || delays[i] > c->max_delay) return fail(c, CFS_EINVAL, "delay outside [0, max_delay]");
    if (c->d_sched) {
      CUDA_TRY(c, cudaStreamSynchronize(c->stream), "schedule");
      dev_free(c, c->d_sched);
      c->d_sched = nullptr;
    }
    c->d_sched = (int8_t*)dev_alloc(c, (size_t)cnt);
    if (!c->d_sched) return fail(c, CFS_ENOMEM, "schedule allocation failed");
    CUDA_TRY(c, cudaMemcpyAsync(c->d_sched, delays, (size_t)cnt, cudaMemcpyHostToDevice, c->stream), "upload schedule");
    CUDA_TRY(c, cudaStreamSynchronize(c->stream), "upload schedule");
    c->sched_steps = nsteps;
  }
  c->algo = algo;
  c->at = at ? 1 : 0;
  c->L = algo == 1 ? L : 1;
  c->graph_dirty = true;
  return CFS_OK;
}

static double* level_ptr(cfs_ctx* c, long long level) { return c->ring + (size_t)(level % c->R) * 5 * c->geo.N; }

cfs_status cfs_set_state(cfs_ctx* c, int block, const double* U, int where) {
  if (!c) return CFS_EINVAL;
  if (!c->finalized) return fail(c, CFS_ESTATE, "set_state after cfs_finalize");
  if (block < 0 || block >= (int)c->blocks.size() || !U) return fail(c, CFS_EINVAL, "bad block or pointer");
  if (c->sticky) return CFS_ECUDA;
  const Block& b = c->blocks[block];
  const size_t bytes = sizeof(double) * 5 * b.N;
  CUDA_TRY(c, cudaMemcpyAsync(level_ptr(c, c->n) + b.base, U, bytes, where ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream), "set_state");
  if (!where) CUDA_TRY(c, cudaStreamSynchronize(c->stream), "set_state");
  return CFS_OK;
}

// The device status word after the stream's work so far (synchronises): a bounded device wait that
// gave up is reported once as CFS_ETIMEOUT and the word is cleared, so the context stays usable.
static cfs_status device_status(cfs_ctx* c) {
  int st = 0;
  CUDA_TRY(c, cudaMemcpyAsync(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "status");
  CUDA_TRY(c, cudaStreamSynchronize(c->stream), "status");
  if (st == 0) return CFS_OK;
  CUDA_TRY(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream), "status");
  return fail(c, CFS_ETIMEOUT, "a bounded device wait gave up (its outputs were set to NaN)");
}

cfs_status cfs_wait_check(cfs_ctx* c, unsigned limit) {
  if (!c) return CFS_EINVAL;
  if (!c->finalized) return fail(c, CFS_ESTATE, "wait check after cfs_finalize");
  if (c->sticky) return CFS_ECUDA;
  const int rc = cfs::launch_wait_check(c->d_status, limit, c->stream);
  if (rc != 0) return cuda_fail(c, (cudaError_t)rc, "wait check launch");
  return CFS_OK;
}

cfs_status cfs_get_state(cfs_ctx* c, int block, double* U, int where) {
  if (!c) return CFS_EINVAL;
  if (!c->finalized) return fail(c, CFS_ESTATE, "get_state after cfs_finalize");
  if (block < 0 || block >= (int)c->blocks.size() || !U) return fail(c, CFS_EINVAL, "bad block or pointer");
  if (c->sticky) return CFS_ECUDA;
  const Block& b = c->blocks[block];
  const size_t bytes = sizeof(double) * 5 * b.N;
  CUDA_TRY(c, cudaMemcpyAsync(U, level_ptr(c, c->n) + b.base, bytes, where ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream), "get_state");
  CUDA_TRY(c, cudaStreamSynchronize(c->stream), "get_state");
  return device_status(c);
}

cfs_status cfs_set_dt(cfs_ctx* c, double dt) {
  if (!c) return CFS_EINVAL;
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, CFS_EINVAL, "dt must be positive");
  c->dt = dt;
  c->dt_set = true;
  c->graph_dirty = true;
  return CFS_OK;
}

cfs_status cfs_get_step(cfs_ctx* c, long long* n) {
  if (!c || !n) return CFS_EINVAL;
  *n = c->n;
  return CFS_OK;
}

cfs_status cfs_set_step(cfs_ctx* c, long long n) {
  if (!c) return CFS_EINVAL;
  if (n < 0) return fail(c, CFS_EINVAL, "negative step");
  c->n = n;
  return CFS_OK;
}

// The sub-domain filter of the FP32 form (all three passes): from the last stage's output to
// level n + 1 (graph mode: the ring slot of the device step counter; the kernel returns on
// synchronous steps, which the per-pass kernels then filter).
static int launch_fblock(cfs_ctx* c, const Geometry& g, const StepSched& sc, const double* src, double* dst, bool graph) {
  cfs::FilterBlockLaunch f{};
  f.Uin = src;
  f.Uout = dst;
  f.ring = c->ring;
  f.in_ring = 0;
  f.out_ring = graph ? 1 : 0;
  f.subs = c->d_subs;
  f.nsub = (int)c->subs.size();
  f.thomas = c->d_thomas;
  f.Lmax = c->Lmax;
  f.alpha = c->p.alpha_f;
  for (int m = 0; m < 6; ++m) f.h[m] = c->filt_h[m];
  f.b1 = c->filt_h[1] - c->p.alpha_f;
  f.halo = c->d_fbhalo;
  const cfs::Timer* tm = (c->timing && !graph) ? &c->timer : nullptr;
  return cfs::launch_filter_block(g, sc, f, c->fblock_n, c->stream, &c->launches, tm);
}

// Exchange of the boundary strips of state array U with the other processes of a partitioned
// context: pack the points the peers read from U, hand both buffers to the caller's transport,
// unpack what arrived into U (the neighbouring PEs' messages of Alg. 1-3).
static cfs_status exchange_strips(cfs_ctx* c, double* U) {
  if (c->part_n <= 1) return CFS_OK;
  if (!c->xfn) return fail(c, CFS_ESTATE, "a partitioned context needs an exchange callback (cfs_set_exchange)");
  int rc = cfs::launch_strip_pack(U, c->d_x_send, c->d_x_send_n, c->x_nsend, c->d_x_sbuf, c->stream);
  if (rc != 0) return cuda_fail(c, (cudaError_t)rc, "strip pack");
  const int xr = c->xfn(c->xuser, c->part_n, c->d_x_sbuf, c->x_send_cnt.data(), c->d_x_rbuf, c->x_recv_cnt.data(),
                        (void*)c->stream);
  if (xr != 0) return fail(c, CFS_EXCHANGE, "the exchange callback reported a failure");
  rc = cfs::launch_strip_unpack(U, c->d_x_recv, c->d_x_recv_n, c->x_nrecv, c->d_x_rbuf, c->stream);
  if (rc != 0) return cuda_fail(c, (cudaError_t)rc, "strip unpack");
  c->launches += 2;
  c->exchanges += 1;
  return CFS_OK;
}

// Enqueue the kernels of step n on the context's stream.  graph = true: the step index and
// everything derived from it (mode, delays, ring slots) are read by the kernels from d_n, so the
// enqueued sequence is the same for every step and can be captured once.
static cfs_status enqueue_step(cfs_ctx* c, long long n, bool graph) {
  const Geometry& g = c->geo;
  const int nops = c->s + (c->p.filter ? c->ndim : 0);
  StepSched sc{};
  sc.n = n;
  sc.R = c->R;
  sc.algo = c->algo;
  sc.L = c->L;
  sc.C = c->C;
  sc.cap = n - c->C + 1;
  sc.mode = (c->algo == 0 || n < c->C) ? 0 : (c->at ? 1 : 2);
  sc.W = c->d_W;
  sc.W32 = c->d_W32;
  sc.W32d = c->d_W32d;
  sc.Wf = c->d_Wf;
  sc.LH = nullptr;
  sc.status = c->d_status;
  sc.table = nullptr;
  sc.at = c->at;
  sc.nsub = (int)c->subs.size();
  sc.table_base = c->algo == 2 ? c->d_sched : nullptr;
  sc.Ntot = g.N;
  sc.dn = graph ? c->d_n : nullptr;
  if (!graph && sc.mode != 0 && c->algo == 2) sc.table = c->d_sched + (size_t)n * c->subs.size() * 6;
  const cfs::Timer* tm = (c->timing && !graph) ? &c->timer : nullptr;
  const double* src = graph ? nullptr : level_ptr(c, n);
  int pp = 0;
  if (c->learned && (graph || sc.mode == 1)) {
    // stage-0 face halos from the network, once per step (the later stages add AT increments)
    const int rc = cfs::launch_mlp_halo(g, sc, c->ring, c->d_subs, c->d_cols, c->ncol, c->d_mlp, c->mlp_scales, c->d_mlpx, c->d_mlpa, c->LH,
                                        c->stream, &c->launches, tm);
    if (rc != 0) return cuda_fail(c, (cudaError_t)rc, "kernel launch");
    sc.LH = c->LH;
  }
  if (c->fused && (graph || sc.mode != 0)) {
    const int rc = cfs::launch_halo_prims(g, c->phys, sc, c->ring, c->d_subs, c->d_halo, c->nhalo, c->Wh, c->s, c->stream,
                                          &c->launches, tm);
    if (rc != 0) return cuda_fail(c, (cudaError_t)rc, "kernel launch");
  }
  for (int op = 0; op < nops; ++op) {
    const bool last_op = op == nops - 1;
    double* dst = last_op ? (graph ? nullptr : level_ptr(c, n + 1)) : c->buf[pp];
    const int in_ring = graph && op == 0, out_ring = graph && last_op;
    int rc;
    // partitioned context, synchronous step: the neighbours' strips of this stage's (or filter
    // pass's) input -- the previous operation's output -- before it is read (Alg. 1)
    if (c->part_n > 1 && sc.mode == 0 && op > 0) {
      const cfs_status xs = exchange_strips(c, const_cast<double*>(src));
      if (xs != CFS_OK) return xs;
    }
    if (op < c->s && c->fused) {
      cfs::FusedLaunch a{};
      a.Uin = src; a.Uout = dst; a.Q = c->Q; a.subs = c->d_subs; a.work = c->d_work; a.nwork = c->nwork;
      a.grid = c->fused_grid; a.fy = c->fused_fy; a.Wh = c->Wh; a.stage = op;
      a.A = c->A[op]; a.B = c->B[op]; a.dt = c->dt; a.first = op == 0; a.last = op == c->s - 1;
      a.ring = c->ring; a.in_ring = in_ring; a.out_ring = out_ring;
      a.curv = c->fused_curv ? 1 : 0;
      rc = cfs::launch_stage_fused(g, c->phys, sc, a, c->stream, &c->launches, tm);
    } else if (op < c->s) {
      cfs::StageLaunch a{};
      a.Uin = src; a.Uout = dst; a.Q = c->Q; a.ring = c->ring; a.subs = c->d_subs;
      a.Wp = c->Wp; a.Phi = c->Phi; a.stage = op; a.s = c->s;
      a.A = c->A[op]; a.B = c->B[op]; a.dt = c->dt;
      a.first = op == 0; a.last = op == c->s - 1;
      a.in_ring = in_ring; a.out_ring = out_ring;
      a.threads = c->threads;
      a.max_pad = c->max_pad; a.max_own = c->max_own; a.max_flux = c->max_flux;
      a.halo = c->d_halo; a.nhalo = c->nhalo;
      a.compact = c->p.compact; a.R = c->Rbuf; a.cthomas = c->d_cthomas; a.Lmax = c->Lmax;
      rc = cfs::launch_stage(g, c->phys, sc, a, c->p.precision, c->stream, &c->launches, tm);
    } else if (op == c->s && c->fblock_n && !graph && sc.mode != 0) {
      // asynchronous step, FP32 form: the three passes in one launch, straight into level n + 1
      rc = launch_fblock(c, g, sc, src, level_ptr(c, n + 1), false);
      if (rc != 0) return cuda_fail(c, (cudaError_t)rc, "kernel launch");
      break;
    } else {
      rc = 0;
      // graph mode: the sub-domain filter (returns on synchronous steps) before the per-pass
      // kernels (which then return on asynchronous steps)
      if (op == c->s && c->fblock_n && graph) rc = launch_fblock(c, g, sc, src, nullptr, true);
      for (const Block& b : c->blocks) {
        if (rc != 0) break;
        cfs::FilterLaunch f{};
        f.Uin = src; f.Uout = dst; f.ring = c->ring;
        f.in_ring = in_ring; f.out_ring = out_ring;
        f.nx = b.nx; f.ny = b.ny; f.nz = b.nz; f.bN = b.N; f.bbase = b.base; f.sid0 = b.sid0;
        f.ebase = b.ebase;
        f.gmx = b.nx + 2 * c->geo.GE;
        f.gmy = b.ny + 2 * c->geo.GE;
        f.wall = f.phys = 0;
        for (int q = 0; q < 6; ++q) {
          if (b.face[q].type >= cfs::FACE_WALL) f.phys |= 1 << q;
          if (b.face[q].type == cfs::FACE_WALL) f.wall |= 1 << q;
        }
        for (int a = 0; a < 3; ++a) {
          f.owner[a] = b.d_owner[a]; f.axis_off[a] = b.d_axis_off[a]; f.axis_len[a] = b.d_axis_len[a];
          f.P[a] = b.P[a];
        }
        f.thomas = c->d_thomas; f.thomas32 = c->d_thomas32; f.Lmax = c->Lmax; f.alpha = c->p.alpha_f;
        {
          const int ax = op - c->s, n3[3] = {b.nx, b.ny, b.nz};
          f.Lt = (n3[ax] + b.P[ax] - 1) / b.P[ax];
        }
        for (int m = 0; m < 6; ++m) f.h[m] = c->filt_h[m];
        f.b1 = c->filt_h[1] - c->p.alpha_f;
        f.only_sync = graph && c->fblock_n;
        f.subs = c->part_n > 1 ? c->d_subs : nullptr;
        rc = cfs::launch_filter(g, sc, f, op - c->s, c->p.precision, c->stream, &c->launches, tm);
        if (rc != 0) break;
      }
    }
    if (rc != 0) return cuda_fail(c, (cudaError_t)rc, "kernel launch");
    src = dst;
    if (!last_op) pp ^= 1;
  }
  if (graph) {
    const int rc = cfs::launch_advance_step(c->d_n, c->stream);
    if (rc != 0) return cuda_fail(c, (cudaError_t)rc, "kernel launch");
    c->launches += 1;
  }
  // partitioned context: publish the boundary strips of U^{n+1} into the neighbours' level n + 1
  // (the send of Alg. 1-3; delayed levels are then read from the ring as on one process)
  if (c->part_n > 1) return exchange_strips(c, level_ptr(c, n + 1));
  return CFS_OK;
}

static cfs_status build_graph(cfs_ctx* c) {
  if (c->gexec) {
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
  }
  cudaGraph_t graph = nullptr;
  CUDA_TRY(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "graph capture");
  const long long before = c->launches;
  cfs_status st = enqueue_step(c, c->n, true);
  cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
  if (st != CFS_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "graph capture");
  c->graph_launches = c->launches - before;
  e = cudaGraphInstantiate(&c->gexec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(c, e, "graph instantiate");
  c->graph_dirty = false;
  return CFS_OK;
}

cfs_status cfs_step(cfs_ctx* c, long long nsteps) {
  if (!c) return CFS_EINVAL;
  if (!c->finalized) return fail(c, CFS_ESTATE, "step after cfs_finalize");
  if (!c->dt_set) return fail(c, CFS_ESTATE, "dt not set");
  if (c->sticky) return CFS_ECUDA;
  if (nsteps < 0) return fail(c, CFS_EINVAL, "negative step count");
  c->launches = 0;
  c->exchanges = 0;
  if (c->algo == 2) {  // asynchronous SAA steps need their rows of the delay table
    const long long last = c->n + nsteps - 1;
    if (nsteps > 0 && last >= c->C && last >= c->sched_steps) {
      // run what the table covers, then report
      const long long ok = std::max(0LL, std::min(nsteps, std::max(c->sched_steps, (long long)c->C) - c->n));
      if (ok > 0) {
        cfs_status st = cfs_step(c, ok);
        if (st != CFS_OK) return st;
      }
      return fail(c, CFS_EINVAL, "step beyond the SAA delay table");
    }
  }
  if (c->graph_on && !c->timing && nsteps > 0) {
    if (c->graph_dirty || !c->gexec) {
      cfs_status st = build_graph(c);
      if (st != CFS_OK) return st;
    }
    CUDA_TRY(c, cudaMemcpyAsync(c->d_n, &c->n, sizeof(long long), cudaMemcpyHostToDevice, c->stream), "step counter");
    for (long long it = 0; it < nsteps; ++it) CUDA_TRY(c, cudaGraphLaunch(c->gexec, c->stream), "graph launch");
    c->n += nsteps;
    c->launches = nsteps * c->graph_launches;
    return CFS_OK;
  }
  for (long long it = 0; it < nsteps; ++it) {
    cfs_status st = enqueue_step(c, c->n, false);
    if (st != CFS_OK) return st;
    c->n += 1;
    if (c->timing && c->ev_used > 4096) timer_flush(c);
  }
  return CFS_OK;
}

cfs_status cfs_set_tiles(cfs_ctx* c, int fy, int zc, int threads) {
  if (!c) return CFS_EINVAL;
  if (c->finalized) return fail(c, CFS_ESTATE, "tiles are set before cfs_finalize");
  if (fy != 4 && fy != 8 && fy != 16) return fail(c, CFS_EINVAL, "tile height must be 4, 8 or 16");
  if (zc < 1 || zc > 4096) return fail(c, CFS_EINVAL, "z chunk must be in 1..4096");
  if (threads != 128 && threads != 256 && threads != 512) return fail(c, CFS_EINVAL, "threads must be 128, 256 or 512");
  c->fused_fy = fy;
  c->fused_zc = zc;
  c->threads = threads;
  return CFS_OK;
}

cfs_status cfs_set_graph(cfs_ctx* c, int on) {
  if (!c) return CFS_EINVAL;
  if (on && c->stream == nullptr) return fail(c, CFS_EINVAL, "graph mode needs a created (non-default) stream");
  if (on && c->part_n > 1) return fail(c, CFS_EINVAL, "a partitioned context steps without a graph (host exchanges)");
  c->graph_on = on != 0;
  c->graph_dirty = true;
  return CFS_OK;
}

cfs_status cfs_set_timing(cfs_ctx* c, int on) {
  if (!c) return CFS_EINVAL;
  if (c->timing) timer_flush(c);
  c->timing = on != 0;
  for (int k = 0; k < CFS_NKINDS; ++k) { c->t_ms[k] = 0.0; c->t_cnt[k] = 0; }
  c->timer.rec = timer_rec;
  c->timer.self = c;
  return CFS_OK;
}

cfs_status cfs_get_timing(cfs_ctx* c, double* ms, long long* count) {
  if (!c) return CFS_EINVAL;
  timer_flush(c);
  for (int k = 0; k < CFS_NKINDS; ++k) {
    if (ms) ms[k] = c->t_ms[k];
    if (count) count[k] = c->t_cnt[k];
  }
  return CFS_OK;
}

cfs_status cfs_diagnostics(cfs_ctx* c, double* out) {
  if (!c || !out) return CFS_EINVAL;
  if (!c->finalized) return fail(c, CFS_ESTATE, "diagnostics after cfs_finalize");
  if (c->sticky) return CFS_ECUDA;
  const double* U = level_ptr(c, c->n);
  int row = 0;
  for (const Block& b : c->blocks) {
    cfs::DiagBlock db{};
    db.nx = b.nx; db.ny = b.ny; db.nz = b.nz; db.bN = b.N; db.bbase = b.base;
    const double a_cd = c->p.order == 4 ? 4.0 / 3.0 : 1.0, b_cd = c->p.order == 4 ? -1.0 / 3.0 : 0.0;
    for (int a = 0; a < 3; ++a) {
      db.c1[a] = (a_cd / 2.0) / b.h[a];
      db.c2[a] = (b_cd / 4.0) / b.h[a];
    }
    db.dV = b.h[0] * b.h[1] * (c->ndim == 3 ? b.h[2] : 1.0);
    db.M = b.mbase >= 0 ? c->d_metric + b.mbase : nullptr;
    db.mx = b.nx + 2 * c->G;
    db.G = c->G;
    db.mpl = (long long)db.mx * (b.ny + 2 * c->G);
    db.rs = c->r;
    db.nonper = 0;
    for (int f = 0; f < 6; ++f)
      if (b.face[f].type != cfs::FACE_PERIODIC) db.nonper |= 1 << f;
    if (db.M)
      for (int a = 0; a < 3; ++a) {  // index-space coefficients
        db.c1[a] = a_cd / 2.0;
        db.c2[a] = b_cd / 4.0;
      }
    if (c->part_n > 1) {  // only the points of the sub-domains computed here
      db.subs = c->d_subs;
      for (int a = 0; a < 3; ++a) {
        db.owner[a] = b.d_owner[a];
        db.P[a] = b.P[a];
      }
      db.sid0 = b.sid0;
    }
    int rc = cfs::launch_diagnostics_block(c->geo, db, U, c->d_partial, row, c->diag_blocks, c->stream);
    if (rc != 0) return cuda_fail(c, (cudaError_t)rc, "diagnostics launch");
    row += c->diag_blocks;
  }
  {
    int rc = cfs::launch_diagnostics_final(c->d_partial, row, c->d_out, c->volume, c->stream);
    if (rc != 0) return cuda_fail(c, (cudaError_t)rc, "diagnostics launch");
  }
  CUDA_TRY(c, cudaMemcpyAsync(out, c->d_out, sizeof(double) * 8, cudaMemcpyDeviceToHost, c->stream), "diagnostics");
  CUDA_TRY(c, cudaStreamSynchronize(c->stream), "diagnostics");
  {
    const cfs_status ds = device_status(c);
    if (ds != CFS_OK) return ds;
  }
  if (out[7] != 0.0) return fail(c, CFS_ENAN, "non-finite value in the state");
  return CFS_OK;
}

cfs_status cfs_eval_power(const double* x, double a, double* y, long long n, void* stream) {
  if (n < 0 || (n > 0 && (!x || !y))) return CFS_EINVAL;
  if (n > (1LL << 40)) return CFS_EINVAL;
  return cfs::launch_eval_power(x, a, y, n, stream) == 0 ? CFS_OK : CFS_ECUDA;
}

cfs_status cfs_fp64_probe(double* sink, int blocks, int iters, void* stream) {
  if (!sink || blocks < 1 || blocks > (1 << 20) || iters < 1) return CFS_EINVAL;
  return cfs::launch_fp64_probe(sink, blocks, iters, stream) == 0 ? CFS_OK : CFS_ECUDA;
}

cfs_status cfs_ring_depth(cfs_ctx* c, int* R) {
  if (!c || !R) return CFS_EINVAL;
  if (!c->finalized) return fail(c, CFS_ESTATE, "ring depth after cfs_finalize");
  *R = c->R;
  return CFS_OK;
}

static cfs_status ring_copy(cfs_ctx* c, double* buf, int where, bool to_ring) {
  const size_t lvl = sizeof(double) * 5 * c->geo.N;
  for (int i = 0; i < c->R; ++i) {
    const long long level = c->n - c->R + 1 + i;
    if (level < 0) continue;
    double* dev = level_ptr(c, level);
    double* other = buf + (size_t)i * 5 * c->geo.N;
    cudaMemcpyKind kind = where ? cudaMemcpyDeviceToDevice : (to_ring ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost);
    CUDA_TRY(c, cudaMemcpyAsync(to_ring ? dev : other, to_ring ? other : dev, lvl, kind, c->stream), "ring copy");
  }
  CUDA_TRY(c, cudaStreamSynchronize(c->stream), "ring copy");
  return CFS_OK;
}

cfs_status cfs_get_ring(cfs_ctx* c, double* buf, int where) {
  if (!c || !buf) return CFS_EINVAL;
  if (!c->finalized) return fail(c, CFS_ESTATE, "ring after cfs_finalize");
  if (c->sticky) return CFS_ECUDA;
  return ring_copy(c, buf, where, false);
}

cfs_status cfs_set_ring(cfs_ctx* c, const double* buf, int where) {
  if (!c || !buf) return CFS_EINVAL;
  if (!c->finalized) return fail(c, CFS_ESTATE, "ring after cfs_finalize");
  if (c->sticky) return CFS_ECUDA;
  return ring_copy(c, const_cast<double*>(buf), where, true);
}

// ------------------------------------------------------------------ learned halo predictor

size_t cfs_mlp_workspace_bytes(long long n) {
  if (n <= 0) return 0;
  return sizeof(float) * (size_t)cfs::mlp_workspace_floats(n);
}

cfs_status cfs_mlp_forward(const float* params, const uint16_t* x, float* y, long long n, void* stream) {
  if (!params || !x || !y || n < 0) return CFS_EINVAL;
  if (n == 0) return CFS_OK;
  return cfs::launch_mlp_forward(params, x, y, n, stream) == 0 ? CFS_OK : CFS_ECUDA;
}

cfs_status cfs_mlp_grad(const float* params, const uint16_t* x, const float* target, long long n, void* workspace,
                        float* grad, float* loss, void* stream) {
  if (!params || !x || !target || !workspace || !grad || n <= 0) return CFS_EINVAL;
  return cfs::launch_mlp_grad(params, x, target, n, (float*)workspace, grad, loss, stream) == 0 ? CFS_OK : CFS_ECUDA;
}

cfs_status cfs_mlp_adamw(float* params, const float* grad, float* m, float* v, int step, float lr, float beta1,
                         float beta2, float eps, float weight_decay, void* stream) {
  if (!params || !grad || !m || !v || step < 1) return CFS_EINVAL;
  return cfs::launch_adamw(params, grad, m, v, MLP_NPARAM, step, lr, beta1, beta2, eps, weight_decay, stream) == 0
             ? CFS_OK
             : CFS_ECUDA;
}

static cfs::MlpScales scales_from(const double* sc) {
  cfs::MlpScales m{};
  for (int v = 0; v < 5; ++v) {
    m.in[v] = sc[v];
    m.own[v] = sc[5 + v];
    m.out[v] = sc[10 + v];
  }
  return m;
}

cfs_status cfs_halo_samples(cfs_ctx* c, const int* spec, long long n, const double* scales, uint16_t* x, float* target,
                            float* at4) {
  if (!c || !spec || !scales || !x || !target || n < 0) return CFS_EINVAL;
  if (!c->finalized) return fail(c, CFS_ESTATE, "samples after cfs_finalize");
  if (c->sticky) return CFS_ECUDA;
  if (c->n < MLP_KMAX + 2 || c->R < MLP_KMAX + 3)
    return fail(c, CFS_ESTATE, "samples need levels n-k-2 for k up to 4 in the ring (n >= 6, max_delay >= 2)");
  if (at4 && (c->p.order != 4 || c->n < MLP_KMAX + c->C - 1 || c->R < MLP_KMAX + c->C || c->max_delay < MLP_KMAX))
    return fail(c, CFS_ESTATE, "AT4 residuals need the fourth-order scheme, max_delay >= 4 and levels n-8..n (n >= 8)");
  StepSched sc{};
  sc.n = c->n;
  sc.R = c->R;
  sc.C = c->C;
  sc.W = c->d_W;
  const int rc = cfs::launch_halo_samples(c->geo, sc, c->ring, c->d_subs, spec, n, scales_from(scales), x, target, at4,
                                          c->s, c->stream);
  if (rc != 0) return cuda_fail(c, (cudaError_t)rc, "samples launch");
  return CFS_OK;
}

cfs_status cfs_set_halo_model(cfs_ctx* c, const float* params, const double* scales, int enable) {
  if (!c) return CFS_EINVAL;
  if (!c->finalized) return fail(c, CFS_ESTATE, "halo model after cfs_finalize");
  if (!enable) {
    c->learned = false;
    c->graph_dirty = true;
    return CFS_OK;
  }
  if (!params || !scales) return fail(c, CFS_EINVAL, "model parameters and scales required");
  if (c->part_n > 1) return fail(c, CFS_EINVAL, "a partitioned context runs the plain AT halos");
  if (!c->all_periodic) return fail(c, CFS_EINVAL, "the halo model needs blocks periodic on every face");
  if (c->max_delay > MLP_KMAX) return fail(c, CFS_EINVAL, "the halo model covers delays 0..4: max_delay must be <= 4");
  if (c->G < MLP_HDEPTH) return fail(c, CFS_EINVAL, "the halo model needs a face halo of depth 4 (viscous CD4)");
  for (int v = 0; v < 15; ++v)
    if (!(scales[v] > 0.0) || !std::isfinite(scales[v])) return fail(c, CFS_EINVAL, "scales must be positive");
  if (!c->d_mlp) {
    std::vector<int> cols;
    const int nsub = (int)c->subs.size();
    for (int sid = 0; sid < nsub; ++sid) {
      const SubDev& d = c->subs[sid];
      const int sz[3] = {d.sx, d.sy, d.sz};
      for (int f = 0; f < 2 * c->ndim; ++f) {
        const int a = f >> 1, b1 = (a + 1) % 3, b2 = (a + 2) % 3;
        for (int t2 = 0; t2 < sz[b2]; ++t2)
          for (int t1 = 0; t1 < sz[b1]; ++t1) {
            cols.push_back(sid); cols.push_back(f); cols.push_back(t1); cols.push_back(t2);
          }
      }
    }
    c->ncol = (long long)(cols.size() / 4);
    c->d_cols = (int*)dev_alloc(c, sizeof(int) * cols.size());
    c->d_mlp = (float*)dev_alloc(c, sizeof(float) * MLP_NPARAM);
    c->LH = (double*)dev_alloc(c, sizeof(double) * 5 * (size_t)c->geo.Ptot);
    const size_t ntile = (size_t)((c->ncol + MLP_TILE - 1) / MLP_TILE);
    c->d_mlpx = (float*)dev_alloc(c, sizeof(float) * ntile * MLP_TILE * MLP_K1);
    c->d_mlpa = (double*)dev_alloc(c, sizeof(double) * ntile * MLP_TILE * MLP_NOUT);
    if (!c->d_cols || !c->d_mlp || !c->LH || !c->d_mlpx || !c->d_mlpa) return fail(c, CFS_ENOMEM, "device allocation failed");
    CUDA_TRY(c, cudaMemcpyAsync(c->d_cols, cols.data(), sizeof(int) * cols.size(), cudaMemcpyHostToDevice, c->stream), "upload columns");
    CUDA_TRY(c, cudaStreamSynchronize(c->stream), "upload columns");
  }
  CUDA_TRY(c, cudaMemcpyAsync(c->d_mlp, params, sizeof(float) * MLP_NPARAM, cudaMemcpyHostToDevice, c->stream), "upload model");
  CUDA_TRY(c, cudaStreamSynchronize(c->stream), "upload model");
  c->mlp_scales = scales_from(scales);
  c->learned = true;
  c->graph_dirty = true;
  return CFS_OK;
}

cfs_status cfs_set_partition(cfs_ctx* c, int nranks, const int* starts, int rank) {
  if (!c) return CFS_EINVAL;
  if (c->finalized) return fail(c, CFS_ESTATE, "partition before cfs_finalize");
  if (nranks < 1 || rank < 0 || rank >= nranks || !starts) return fail(c, CFS_EINVAL, "bad partition");
  if (starts[0] != 0) return fail(c, CFS_EINVAL, "the partition starts at sub-domain 0");
  for (int q = 0; q < nranks; ++q)
    if (starts[q + 1] < starts[q]) return fail(c, CFS_EINVAL, "partition boundaries must not decrease");
  if (nranks > 1 && c->graph_on) return fail(c, CFS_EINVAL, "a partitioned context steps without a graph");
  c->part_n = nranks;
  c->part_rank = rank;
  c->part_starts.assign(starts, starts + nranks + 1);
  return CFS_OK;
}

cfs_status cfs_set_exchange(cfs_ctx* c, cfs_exchange_fn fn, void* user) {
  if (!c) return CFS_EINVAL;
  c->xfn = fn;
  c->xuser = user;
  return CFS_OK;
}

cfs_status cfs_exchange_plan(cfs_ctx* c, int peer, int which, long long* offsets, long long* count) {
  if (!c || !count || (which != 0 && which != 1)) return CFS_EINVAL;
  if (c->part_n <= 1) return fail(c, CFS_ESTATE, "no partition set");
  if (peer < 0 || peer >= c->part_n) return fail(c, CFS_EINVAL, "peer out of range");
  std::vector<cfs::TopoBlock> topo;
  if (const char* why = host_topology(c, topo)) return fail(c, CFS_EINVAL, why);
  int nsub = 0;
  for (const Block& b : c->blocks) nsub += b.P[0] * b.P[1] * b.P[2];
  if ((int)c->part_starts.size() != c->part_n + 1 || c->part_starts[c->part_n] != nsub)
    return fail(c, CFS_EINVAL, "the partition does not cover the sub-domains");
  const int need = c->p.filter ? (c->G > 5 ? c->G : 5) : c->G;
  cfs::StripPlan plan;
  if (const char* why = cfs::strip_plan(topo.data(), (int)topo.size(), nsub, c->part_starts.data(), c->part_n,
                                        c->part_rank, need, c->ndim == 3 ? need : 0, c->r, c->p.viscous != 0, c->ndim,
                                        &plan))
    return fail(c, CFS_EINVAL, why);
  const std::vector<long long>& off = which == 0 ? plan.send_off : plan.recv_off;
  const std::vector<long long>& lst = which == 0 ? plan.send : plan.recv;
  *count = off[peer + 1] - off[peer];
  if (offsets)
    for (long long i = 0; i < *count; ++i) offsets[i] = lst[off[peer] + i];
  return CFS_OK;
}

cfs_status cfs_exchange_count(cfs_ctx* c, long long* n) {
  if (!c || !n) return CFS_EINVAL;
  *n = c->exchanges;
  return CFS_OK;
}

cfs_status cfs_launch_count(cfs_ctx* c, long long* launches) {
  if (!c || !launches) return CFS_EINVAL;
  *launches = c->launches;
  return CFS_OK;
}

const char* cfs_last_error(cfs_ctx* c) {
  if (!c) return kNoCtx;
  return c->err.c_str();
}

void cfs_destroy(cfs_ctx* c) {
  if (!c) return;
  if (c->finalized) cudaStreamSynchronize(c->stream);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  for (void* q : c->owned) c->freef(q, c->user);
  c->owned.clear();
  delete c;
}

}  // extern "C"
