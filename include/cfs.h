/*
 * cfs.h -- C ABI of the GB300 asynchronous compressible flow solver library (libcfs.so).
 *
 * The library advances the compressible Navier-Stokes (or Euler) equations on blocks -- uniform
 * Cartesian or curvilinear (App. A), periodic or joined by interfaces and bounded by walls, far
 * fields and outflows (a multi-block grid such as the airfoil C-grid of Sec. 5.3) -- split into
 * sub-domains ("processing elements" of arXiv 2506.03027, Sec. 3), with the asynchrony-tolerant
 * (AT) halo treatment of Sec. 3.1-3.2 under the SA, CAA and SAA algorithms of Alg. 1-3.  Every step of the hot path runs in the library's CUDA kernels for
 * sm_103a; there is no CPU fallback: a call that needs the GPU fails with CFS_ECUDA when the
 * device or the kernels are unavailable.
 *
 * Conventions
 *   - State arrays are structure-of-arrays FP64, U[5][nz][ny][nx] with x fastest, variables
 *     {rho, rho u, rho v, rho w, rho E_t} (Eq. 1).  2-D runs use nz = 1 and rho w = 0.
 *   - Pointers are plain host or device addresses as stated per call; sizes are element counts.
 *   - The library never frees memory it did not allocate.  Device memory comes from the
 *     allocator set with cfs_set_allocator (default: cudaMalloc / cudaFree).
 *   - All device work is issued on the stream passed to cfs_create (borrowed, not owned).
 *     Calls that return data to the host synchronise that stream.
 *   - Errors: every call returns a cfs_status; cfs_last_error gives a message.  A CUDA error is
 *     sticky for the context.  No C++ exception crosses this interface.
 */
#ifndef CFS_H_
#define CFS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CFS_OK = 0,
  CFS_EINVAL = 1,   /* invalid argument (sizes, schedule, scheme) */
  CFS_ENOMEM = 2,   /* the allocator returned NULL */
  CFS_ECUDA = 3,    /* CUDA runtime error (sticky) */
  CFS_ESTATE = 4,   /* call out of order (e.g. cfs_step before cfs_finalize) */
  CFS_ENAN = 5,     /* non-finite value found in the state */
  CFS_ETIMEOUT = 6, /* a bounded device wait gave up */
  CFS_EXCHANGE = 7  /* the exchange callback of a partitioned context reported a failure */
} cfs_status;

typedef struct cfs_ctx cfs_ctx;

/* Scheme and physics (Table 1, App. A-B).  Nondimensionalisation of App. A:
 * E_t = T/(gamma (gamma-1) M^2) + |u|^2/2, p = rho T/(gamma M^2), viscous terms scaled by 1/Re,
 * heat flux mu/((gamma-1) Pr M^2) dT/dx. */
typedef struct {
  int order;         /* 4: LSERK4-CD4-AT4 (5 stages, C = 5 levels); 2: LSERK2-CD2-AT2 (2, 3) */
  int viscous;       /* 1: Navier-Stokes (Eq. A3-A4), 0: Euler */
  int visc_law;      /* 0: mu = 1; 1: mu = T^visc_exp */
  double visc_exp;
  double gamma, mach, re, pr;
  int filter;        /* 1: tenth-order Pade filter (coefficient alpha_f) once per step */
  double alpha_f;
  int precision;     /* 0: FP64 throughout; 1: FP32 derivative/flux/filter intermediates with
                        FP64 state and RK accumulation; the AT halo values are summed to FP64
                        accuracy (compensated FP32 sums over the delayed levels' differences,
                        FP64 sums for the filter halos) before their rounding to FP32 */
  int compact;       /* 1: the flux divergence by the sixth-order compact scheme of Eq. 2 (alpha =
                        1/3, a = 14/9, b = 1/9), one tridiagonal solve per sub-domain line, closed by
                        the explicit sixth-order central difference at the first halo point (halo
                        depth 4); Euler (viscous = 0) with order 4 (LSERK4, AT4) on Cartesian
                        blocks periodic on every face, FP64 (precision 0) only; 0: explicit CD */
} cfs_params;

/* Device allocator used by cfs_finalize and cfs_set_schedule.  alloc returns a device pointer
 * aligned to at least 256 bytes or NULL; free releases it. */
typedef void* (*cfs_alloc_fn)(size_t bytes, void* user);
typedef void (*cfs_free_fn)(void* ptr, void* user);

/* Create a context.  p is copied.  cuda_stream is a cudaStream_t (NULL = legacy default stream)
 * that the caller keeps alive until cfs_destroy.  *out receives the context.
 * EINVAL: unsupported order/precision/filter coefficient (|alpha_f| must be < 0.5). */
cfs_status cfs_create(const cfs_params* p, void* cuda_stream, cfs_ctx** out);

/* Replace the device allocator (before cfs_finalize).  user is passed back unchanged. */
cfs_status cfs_set_allocator(cfs_ctx* ctx, cfs_alloc_fn alloc, cfs_free_fn free_fn, void* user);

/* Add a uniform Cartesian block of ni x nj x nk points with spacing {dx, dy, dz} (host array of
 * 3 doubles), periodic in every direction until connected (cfs_connect) or bounded (cfs_set_bc).
 * nk = 1 makes the run two-dimensional.  *block_id receives the index (0, 1, ... in the order of
 * the calls).  Several blocks of uneven sizes advance together -- independent problems, or one
 * connected grid: every stage launch covers the sub-domains of all blocks, whose states are
 * stored one after another (block b at offset 5 x the points of blocks 0..b-1 in a state array).
 * All blocks share the physics, scheme, dt and schedule algorithm; they must all be 2-D or all
 * 3-D.  EINVAL for non-positive sizes or mixed dimensionality. */
cfs_status cfs_add_block(cfs_ctx* ctx, int ni, int nj, int nk, const double* spacing, int* block_id);

/* Make block `block` curvilinear (App. A: Eq. A1 in strong conservation form on general
 * coordinates, fluxes of Eq. A2 with contravariant velocities, viscous terms of Eq. A3-A4 with
 * the chain rule through the metric terms).  The grid is a smooth mapping of the index plane
 * (i, j) extruded along z: xy is a HOST array [2][nj][ni] with x(i, j) then y(i, j); z = k dz
 * with dz the block's third spacing (unit depth in 2-D).  Across a periodic face shift[0..1] is
 * the (x, y) jump of the coordinates across the wrap in i, shift[2..3] the jump across the wrap
 * in j (for example (Lx, 0, 0, Ly) for a deformed rectangle); across an interface the grid
 * continues into the neighbour, across a physical boundary it is reflected (cfs_set_bc).  At cfs_finalize the library computes the metric terms xi^_x = J^-1 dxi/dx ...
 * and J from the coordinates with the block's own CD scheme in index space (their cofactor
 * form keeps a uniform flow uniform to rounding); derivatives of the solution are then taken
 * in index space.  The data are copied.  Call after cfs_add_block, before cfs_finalize
 * (ESTATE otherwise); EINVAL for an unknown block, null pointers or non-finite values, and at
 * cfs_finalize for a grid with a non-positive cell volume.  The FP32-intermediate precision runs
 * 3-D Navier-Stokes CD4 on curvilinear blocks -- periodic or connected (interfaces, walls, far
 * fields, outflows) -- through the fused stage (one launch per RK stage). */
cfs_status cfs_set_block_grid(cfs_ctx* ctx, int block, const double* xy, const double* shift);

/* Decompose a block into pi x pj x pk sub-domains (the paper's PEs, Sec. 3); sub-domains are
 * numbered block after block, x fastest within a block.  Along each axis
 * n points split into p parts as evenly as possible, the first n mod p parts one point longer.
 * Every sub-domain must be at least as wide as the halo it needs (2 r for viscous runs, r for
 * Euler, r = 2 for CD4 and 1 for CD2; 5 with the filter).  EINVAL otherwise. */
cfs_status cfs_split_block(cfs_ctx* ctx, int block, int pi, int pj, int pk);

/* Connect face faceA of blockA to faceB of blockB (faces 0..5 = -i,+i,-j,+j,-k,+k) -- the
 * block interfaces of a multi-block grid such as the paper's airfoil C-grid (Sec. 5.3), whose
 * topology the paper does not print.  Every face is periodic (self-connected) until connected or
 * bounded.  The same block and opposite faces with orientation 0 restore the periodic default.
 * Otherwise both faces must be x or y faces (blocks are extruded and periodic in z); the blocks
 * are node-disjoint: the first point beyond faceA is blockB's first point inside faceB.
 * orientation 0: the tangential in-plane index runs the same way on both sides; 1: reversed
 * (a C-grid's wake cut joins the -j faces of its two wake blocks this way).  The tangential point
 * counts must match (checked at cfs_finalize); spanwise counts may differ: a point then takes the
 * neighbour's values at its own spanwise position by four-point Lagrange interpolation.
 * Curvilinear blocks join only curvilinear blocks; two Cartesian blocks only opposite faces of
 * one axis, unreversed.  Halo values across an interface are the neighbouring PE's values, seen
 * with the face's delay (Alg. 2-3).  ESTATE after cfs_finalize, EINVAL on a bad argument. */
cfs_status cfs_connect(cfs_ctx* ctx, int blockA, int faceA, int blockB, int faceB, int orientation);

/* Coordinate jump (x, y) added to the neighbour's point coordinates when the grid of a
 * curvilinear block is continued across interface `face` (nonzero where an interface closes a
 * periodic direction).  Call after cfs_connect; EINVAL if the face is not an interface. */
cfs_status cfs_set_face_shift(cfs_ctx* ctx, int block, int face, const double* shift);

/* The sources of the state the kernels take at point (i, j, k) of `block`'s index space (a point
 * up to the halo depth beyond its faces), for inspecting a multi-block description: the faces are
 * validated as at cfs_finalize (which need not have been called).  out[34] (host): out[0] the
 * number of sources (up to 4), out[1..5] the far-field constant added to the conserved values,
 * then per source 7 values: block, i, j, k, weight, mirrored (momentum negated), crossed (reached
 * through a periodic wrap or an interface: a neighbouring PE's value).  Value v of the point =
 * out[1 + v] + sum over sources of weight * (mirrored and 1 <= v <= 3 ? -1 : 1) * U_v(source).
 * EINVAL for a bad block, a point beyond the halo depth or an invalid face description. */
cfs_status cfs_halo_sources(cfs_ctx* ctx, int block, int i, int j, int k, double* out);

/* The metric terms the kernels use at point (i, j) of curvilinear `block`'s plane (up to the halo
 * depth beyond its faces; blocks are extruded, so every z has the same): out[7] (host) =
 * {xi^_x, xi^_y, eta^_x, eta^_y, zeta^_z, J^-1, J} of App. A, from the grid continued across the
 * faces (NaN beyond a non-periodic face deeper than the stencil radius, where no flux is
 * evaluated).  For inspecting a grid before cfs_finalize; EINVAL for a Cartesian or unknown
 * block, a point beyond the halo depth, an invalid face description or a grid with a
 * non-positive cell volume. */
cfs_status cfs_metric_terms(cfs_ctx* ctx, int block, int i, int j, double* out);

/* Physical boundary condition on x or y face `face` of `block`:
 *   CFS_BC_WALL      no-slip adiabatic wall: the points on the face are wall points, whose
 *                    momentum is held at zero; beyond the face the state is mirrored about it
 *                    with the momentum negated (data unused);
 *   CFS_BC_FARFIELD  the conserved state data[5] (host, copied) beyond the face;
 *   CFS_BC_OUTFLOW   the face values repeated beyond it (data unused);
 *   CFS_BC_PERIODIC  the face and its opposite face periodic again.
 * These halo closures are readings: the paper does not print its boundary treatment.  Beyond a
 * physical face the grid of a curvilinear block is reflected through the boundary point.  A halo
 * source reached by a wall mirror or an outflow copy inside the same sub-domain is the PE's own
 * current value for points inside the sub-domain along z; beyond a z face such a source is
 * reached across the periodic wrap (or lies in the z-neighbour) and is seen with that face's
 * delay.  Before cfs_finalize (ESTATE after); EINVAL on a bad argument. */
#define CFS_BC_PERIODIC 0
#define CFS_BC_WALL 1
#define CFS_BC_FARFIELD 2
#define CFS_BC_OUTFLOW 3
cfs_status cfs_set_bc(cfs_ctx* ctx, int block, int face, int type, const double* data);

/* Allocate device memory for the state ring, stage buffers and scratch, and build the
 * sub-domain tables.  max_delay is the largest delay any schedule will use (sizes the ring of
 * delayed levels: max_delay + C + 1 full states).  ESTATE if called twice, ENOMEM on
 * allocation failure. */
cfs_status cfs_finalize(cfs_ctx* ctx, int max_delay);

/* Delay schedule (Alg. 1-3).  algo: 0 SA, 1 CAA, 2 SAA.  at: 1 AT schemes, 0 AS (standard
 * stencils on the latest delayed level).  The first C steps of CAA/SAA run synchronously.
 *   CAA: delay of every face at step n >= C is (n - C) mod L (L >= 1, L - 1 <= max_delay).
 *   SAA: delays is a HOST table int8[nsteps][nsub][6] (step, sub-domain, face), copied; each
 *        entry must lie in [0, max_delay].  Steps beyond nsteps are an error at cfs_step.
 * Delays are clamped to n - C + 1 so that every referenced level exists.  Sub-domains are
 * numbered x fastest.  EINVAL on out-of-range entries. */
cfs_status cfs_set_schedule(cfs_ctx* ctx, int algo, int at, int L, long long nsteps, const int8_t* delays);

/* Copy the state of block `block` ([5][nz][ny][nx] of that block) in (set) or out (get).
 * where: 0 = host pointer, 1 = device pointer.  set_state defines the state at the current step index (0 after cfs_finalize; see
 * cfs_set_step) and is the start of a fresh history unless the ring is restored as well.
 * get_state synchronises the stream; it returns ETIMEOUT (with the state copied) when a bounded
 * device wait gave up since the last report (cfs_wait_check). */
cfs_status cfs_set_state(cfs_ctx* ctx, int block, const double* U, int where);
cfs_status cfs_get_state(cfs_ctx* ctx, int block, double* U, int where);

/* Fixed time step (the AT weights assume equally spaced levels, Eq. 5 and Eq. 9). */
cfs_status cfs_set_dt(cfs_ctx* ctx, double dt);

/* Current step index n (levels U^0..U^n exist).  cfs_set_step moves it (with cfs_set_ring for
 * checkpoint / resume). */
cfs_status cfs_get_step(cfs_ctx* ctx, long long* n);
cfs_status cfs_set_step(cfs_ctx* ctx, long long n);

/* Advance nsteps time steps: per step, s LSERK stages of the fused RHS + stage update with the
 * halos of the schedule, then the filter (if on); the new state is U^{n+1}.  Asynchronous on the
 * stream; errors of device work surface at the next synchronising call. */
cfs_status cfs_step(cfs_ctx* ctx, long long nsteps);

/* Launch shapes (before cfs_finalize): tile height fy (4, 8 or 16) and z chunk zc of the fused
 * FP32-intermediate stage kernel (tiles of 32 x fy columns marching zc planes), and the threads per
 * CTA (128, 256, 512) of the other stage kernels; defaults 16, 32 and 256.  Results are identical
 * for every choice; the autotuner of the Python package picks the fastest and stores it. */
cfs_status cfs_set_tiles(cfs_ctx* ctx, int fy, int zc, int threads);

/* CUDA-graph mode (on = 1): cfs_step captures the kernels of one step once -- the step index is
 * kept in device memory and every kernel derives the step's mode, delays and ring slots from it --
 * and replays the graph once per step.  The graph is rebuilt after cfs_set_dt, cfs_set_schedule
 * or cfs_set_halo_model.  Needs a created (non-default) stream: EINVAL for the legacy stream.
 * Per-kernel timing (cfs_set_timing) bypasses the graph. */
cfs_status cfs_set_graph(cfs_ctx* ctx, int on);

/* Self-test of the bounded device waits (no counterpart in the paper: a check of the library's
 * failure reporting).  The tensor-core kernels wait on mbarriers with a poll limit; a wait that gives
 * up sets a status word of the context (and poisons that kernel's outputs with NaN), which the next
 * synchronising call that returns data -- cfs_get_state, cfs_diagnostics -- reports once as
 * CFS_ETIMEOUT, after which the context stays usable.  This call launches, on the context's stream,
 * one CTA that waits on an mbarrier nothing arrives at, gives up after `limit` polls and sets the
 * word.  ESTATE before cfs_finalize. */
cfs_status cfs_wait_check(cfs_ctx* ctx, unsigned limit);

/* Diagnostics of the current state U^n over all blocks (synchronises): out[8] = {K, enstrophy,
 * sum rho, sum rho u, sum rho v, sum rho w, sum rho E, non-finite flag}, K and enstrophy point averages
 * with rho_0 = 1 (Sec. 5.2), vorticity by the scheme's central difference, sums weighted by the
 * cell volume.  The enstrophy average covers the points whose difference stencils stay inside their
 * block or cross only periodic faces.  Returns ENAN (and fills out) when the state holds a
 * non-finite value, ETIMEOUT (and fills out) when a bounded device wait gave up since the last
 * report (cfs_wait_check). */
cfs_status cfs_diagnostics(cfs_ctx* ctx, double* out);
/* (On a partitioned context the diagnostics cover the points of the sub-domains computed here:
 * K, the totals and the non-finite flag combine over the processes by sums and a max; the
 * enstrophy is the average over this process's points.) */

/* The library's FP64 power y[i] = x[i]^a for n device values, asynchronously on `stream` (the
 * power-law viscosity mu = T^a of App. A's constitutive law, as the FP64 path evaluates it: a
 * table-driven logarithm and exponential of about 20 FP64 operations; for positive normal x its
 * relative error is below 6e-16 (1 + |a ln x|), 1.2e-15 for x near 1).  For checking that power against
 * a reference; EINVAL for a negative n or null buffers, ECUDA if the launch fails. */
cfs_status cfs_eval_power(const double* x, double a, double* y, long long n, void* stream);

/* Measurement aid (no counterpart in the paper): the FP64 pipe rate that the FP64 path's roofline
 * divides by.  Launches `blocks` CTAs of 256 threads, each thread running 8 independent FP64 FMA
 * chains of `iters` steps, and writes one value per thread to sink (device, blocks x 256 doubles,
 * caller-owned), asynchronously on `stream`.  FMAs executed = blocks x 256 x iters x 8 (2 flops
 * each); the caller times the launch.  EINVAL for a null sink, blocks outside 1..2^20 or
 * iters < 1; ECUDA if the launch fails. */
cfs_status cfs_fp64_probe(double* sink, int blocks, int iters, void* stream);

/* Checkpoint / resume of the ring of delayed levels: R = max_delay + C + 1 full states,
 * slot i holds level n - R + 1 + i (host or device buffer of R * 5 * npoints doubles). */
cfs_status cfs_ring_depth(cfs_ctx* ctx, int* R);
cfs_status cfs_get_ring(cfs_ctx* ctx, double* buf, int where);
cfs_status cfs_set_ring(cfs_ctx* ctx, const double* buf, int where);

/* Host-side coefficient tables generated by the library (no GPU needed), for inspection:
 * W[(k * s + m) * C + l] = weight of level n-k-l in the stage-m halo value (m = 0: Eq. 14/15
 * extrapolation; m >= 1: after the buffer updates of Eq. 8 at stages 1..m), k = 0..kmax.
 * Returns the number of doubles written (kmax+1)*s*C, or -1 on bad arguments. */
int cfs_at_weights(int order, int kmax, double* W);

/* ------------------------------------------------------------------ partitioned contexts
 * The paper's PEs (Sec. 3) spread over processes (one GPU each): every process creates a context
 * for the whole grid, with the same blocks, splits, physics and schedule, and computes a
 * contiguous range of sub-domains.  The only data that travel are the boundary strips of the
 * new solution that neighbouring PEs read (Alg. 1-3: the send of U^{n+1} at the end of every step
 * into the neighbours' delayed levels, and under SA -- also the synchronous warm-up steps of CAA
 * and SAA -- the strips of every stage's and filter pass's input).  A process keeps state arrays
 * of the whole grid; points of other processes' sub-domains hold the strips it received (the
 * rest of them is never read and keeps whatever cfs_set_state or cfs_set_ring wrote).  The
 * delays stay those of the schedule, so a partitioned run gives bit for bit the results of one
 * context computing every sub-domain. */

/* Compute sub-domains [starts[rank], starts[rank + 1]) of the nranks ranges in starts[nranks + 1]
 * (host, copied; starts[0] = 0, non-decreasing, starts[nranks] = the number of sub-domains, checked
 * at cfs_finalize).  Before cfs_finalize (ESTATE after).  nranks = 1 restores the single-process
 * context.  Periodic blocks and connected grids (interfaces, walls, far fields, outflows: the
 * sources of the points beyond their faces travel like any other halo point).  At cfs_finalize
 * EINVAL unless the precision is FP64 (0); the learned halo and CUDA-graph mode are refused on a
 * partitioned context. */
cfs_status cfs_set_partition(cfs_ctx* ctx, int nranks, const int* starts, int rank);

/* Transport of a partitioned context, called by cfs_step at every exchange point with:
 * send (device) -- the packed strips for every peer, peer q's send_counts[q] doubles starting at
 * the sum of send_counts[0..q-1]; recv (device) -- room for what every peer sends here, laid out
 * the same way with recv_counts; nranks; and the context's stream.  The packing is enqueued on
 * that stream: the callback orders its reads after it (cudaStreamSynchronize, or transfers
 * enqueued on the stream such as NCCL send/recv), and before returning has the received values in
 * recv, or enqueued on the stream ahead of anything enqueued later.  Counts to and from the own
 * rank are 0.  Layout of a peer's part: 5 doubles (rho, rho u, rho v, rho w, rho E) per point, points
 * in the order of cfs_exchange_plan.  Return 0 on success; anything else makes cfs_step fail with
 * CFS_EXCHANGE. */
typedef int (*cfs_exchange_fn)(void* user, int nranks, const double* send, const long long* send_counts, double* recv,
                               const long long* recv_counts, void* stream);
cfs_status cfs_set_exchange(cfs_ctx* ctx, cfs_exchange_fn fn, void* user);

/* The exchange plan of a partitioned context (host; cfs_finalize need not have been called):
 * which = 0 the points this rank sends to `peer` -- its own points that peer's sub-domains read
 * (faces to the halo depth, 5 with the filter, viscous edges to r x r) --, which = 1 those it
 * receives from peer.  *count receives the number of points; offsets (host, may be NULL) receives
 * their state offsets (block base + point index; variable v at + v x the block's points), sorted.
 * Rank p's send list to q equals rank q's receive list from p.  ESTATE without a partition. */
cfs_status cfs_exchange_plan(cfs_ctx* ctx, int peer, int which, long long* offsets, long long* count);

/* Exchange callbacks made by the last cfs_step call. */
cfs_status cfs_exchange_count(cfs_ctx* ctx, long long* n);

/* Counters of the last cfs_step call: number of kernel launches issued. */
cfs_status cfs_launch_count(cfs_ctx* ctx, long long* launches);

/* Per-kernel timing with CUDA events recorded on the context's stream around every launch.
 * cfs_set_timing(ctx, 1) starts (and clears) the accumulation, 0 stops it.  cfs_get_timing
 * synchronises and returns, for each kernel kind k (CFS_NKINDS entries: 0 view, 1 flux,
 * 2 stage update, 3 filter, 4 diagnostics), the summed duration ms[k] in milliseconds and the
 * number of timed launches count[k].  Either array may be NULL. */
#define CFS_NKINDS 5
cfs_status cfs_set_timing(cfs_ctx* ctx, int on);
cfs_status cfs_get_timing(cfs_ctx* ctx, double* ms, long long* count);

/* ------------------------------------------------------------------ learned halo predictor
 * A 3-layer perceptron (CFS_MLP_NIN -> 64 -> 64 -> CFS_MLP_NOUT, GELU in tanh form) predicts for
 * one face column of a sub-domain's halo (4 points deep, 5 variables) the residual of the current
 * level over the 3-level extrapolation of Eq. 14, from BF16 features of the delayed levels:
 *   x[0..19]   (U^{n-k} - U^{n-k-1}) * in_scale[v] at the 4 halo points,
 *   x[20..39]  (U^{n-k-1} - U^{n-k-2}) * in_scale[v],
 *   x[40..59]  (U^n - U^{n-k}) * own_scale[v] at the 4 own points next to the face,
 *   x[60..64]  one-hot delay k (0..4),
 * each rounded FP64 -> FP32 (to nearest) -> BF16 (to nearest even), index (depth - 1) * 5 + v.
 * Output y[(depth - 1) * 5 + v] = (U^n - extrapolation) * out_scale[v].  Parameters are FP32:
 * W1[64][65], b1[64], W2[64][64], b2[64], W3[20][64], b3[20] (CFS_MLP_NPARAM floats).  The paper has
 * no counterpart: this is the learned form of the halo, compared against the plain AT stencil. */
#define CFS_MLP_NIN 65
#define CFS_MLP_NOUT 20
#define CFS_MLP_NPARAM 9684

/* Forward pass: y[n][20] (device, FP32) from x[n][65] (device, BF16 bit patterns) and params
 * (device).  Asynchronous on stream. */
cfs_status cfs_mlp_forward(const float* params, const uint16_t* x, float* y, long long n, void* stream);

/* Bytes of the caller-provided device workspace cfs_mlp_grad needs for n samples. */
size_t cfs_mlp_workspace_bytes(long long n);

/* Gradient of the mean squared error mean((y - target)^2) over n samples and 20 outputs with
 * respect to all parameters into grad (device, CFS_MLP_NPARAM floats) and the loss into *loss
 * (device float, may be NULL).  Deterministic: per-chunk sums in a fixed order, then chunk order. */
cfs_status cfs_mlp_grad(const float* params, const uint16_t* x, const float* target, long long n, void* workspace,
                        float* grad, float* loss, void* stream);

/* One AdamW update (decoupled weight decay, bias-corrected moments) of all parameters; m and v are
 * the caller's device moment buffers; step counts from 1. */
cfs_status cfs_mlp_adamw(float* params, const float* grad, float* m, float* v, int step, float lr, float beta1,
                         float beta2, float eps, float weight_decay, void* stream);

/* Training samples from the context's ring at its current step n (a synchronous run gives the true
 * current halo values): spec (device int32 [n][5]) = (sub-domain, face 0..5, t1, t2, delay k) with
 * t1, t2 the owned coordinates along the axes (a+1)%3 and (a+2)%3 of the face's axis a; scales
 * (host, 15 doubles: in_scale[5], own_scale[5], out_scale[5]); writes x (device BF16 [n][65]) and
 * target (device FP32 [n][20]).  Needs n >= 6 and a ring that holds levels n-6..n.  at4 (device FP32
 * [n][20], or NULL): the residual of the AT4 stage-0 halo value of Eq. 15 -- the five-level
 * extrapolation with c(k) from levels n-k .. n-k-4 -- over the true value, times out_scale, the
 * same units as target: the error of the method the network replaces (needs the fourth-order
 * scheme, max_delay >= 4 and n >= 8). */
cfs_status cfs_halo_samples(cfs_ctx* ctx, const int* spec, long long n, const double* scales, uint16_t* x, float* target,
                            float* at4);

/* Use (enable = 1) or stop using (0) the network for the stage-0 face halos of AT steps: each step,
 * every face column's U_buf^(0) = extrapolation + y / out_scale; later stages add the AT buffer-update
 * increments (W^(m) - W^(0)) R.  Edge halos keep the AT weights.  params and scales are host arrays,
 * copied.  EINVAL if max_delay > 4 or the run is not viscous CD4 (face halo depth 4). */
cfs_status cfs_set_halo_model(cfs_ctx* ctx, const float* params, const double* scales, int enable);

/* Diagnostics without any device allocation (no counterpart in the paper: an interface for
 * callers that cannot allocate).  Callers such as an in-situ monitoring hook inside a larger
 * simulation whose pool allocator owns all of the GPU's memory, or a time-critical loop where an
 * allocation (which may synchronise the device) is not allowed, cannot use cfs_diagnostics,
 * whose context allocates its scratch at cfs_finalize.  This call computes the same eight
 * quantities for a state U (device pointer, FP64 [5][nz][ny][nx], periodic grid with spacing
 * {dx, dy, dz} given as a host array of 3 doubles, CD scheme of `order` 2 or 4 for the vorticity)
 * and writes them to out (device pointer to 8 doubles), asynchronously on cuda_stream.
 *   - Scratch: a fixed array of per-block partial sums compiled into the library (4 MiB, kept on
 *     every GPU that loads the library until the process exits).  It limits the grid to
 *     CFS_DIAG_STATIC_MAX_POINTS points; larger grids are rejected with CFS_EINVAL and a message.
 *   - No cudaMalloc, cudaFree or other allocating call is made.
 *   - The first call on each device (with that device current) looks up the array's device
 *     address and keeps it for the life of the process; make that first call before any stream
 *     capture.  The kept address is not valid across a reset of the device (cudaDeviceReset):
 *     do not call this entry point in a process after resetting the device it runs on.
 *   - All calls share the array; each call overwrites the partial sums it reads, so nothing has
 *     to be cleared, but calls whose GPU work overlaps (other streams, other host threads) race.
 *   - err (may be NULL) receives a message of at most err_len bytes on failure.
 * Returns CFS_OK, CFS_EINVAL (bad pointer, size or order) or CFS_ECUDA (device or launch error). */
#define CFS_DIAG_STATIC_MAX_POINTS 16777216LL
cfs_status cfs_diagnostics_static(const double* U, int nx, int ny, int nz, const double* spacing, int order,
                                  double* out, void* cuda_stream, char* err, size_t err_len);

/* Last error message of the context (static string if ctx is NULL). */
const char* cfs_last_error(cfs_ctx* ctx);

/* Release device memory (through the allocator) and the context. */
void cfs_destroy(cfs_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* CFS_H_ */
