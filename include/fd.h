/*
 * fd.h -- C ABI of the B300 finite-difference time-stepping library.
 *
 * One context (fd_ctx) holds one simulation on one GPU: a structured 2-D or
 * 3-D grid, its time levels and model coefficients in HBM, optional point
 * sources and receivers, and a CUDA stream.  The calls follow the problem
 * statement of a Devito operator (thesis §2.1.1: Grid(shape, extent),
 * TimeFunction(time_order, space_order), initial data written into u.data[0],
 * sparse functions for sources and receivers, op(time=nt, dt=dt)) and the
 * benchmark problem of §5.1.2.
 *
 * Equations (L = Σ_d (1/h_d²) Σ_{k=-r..r} w_|k| shift_d^k, r = space_order/2,
 * w = central second-derivative weights of order space_order; outside the grid
 * every field is zero):
 *
 *   FD_DIFFUSION  (§5.1.2, u_t = ν Σ_d u_dd, forward Euler, time order 1):
 *       u^{n+1} = u^n + ν dt L u^n     on interior nodes (index 1..n_d-2 on
 *       every axis, §2.1.1's grid.interior); boundary nodes keep the values
 *       given to fd_set_field (fd_options.dirichlet_interior = 0: on every node).
 *   FD_ACOUSTIC   (the seismic operator of §6.2.1, m u_tt + damp u_t = L u + src,
 *       second-order leapfrog on every node, σ = damp·dt/2):
 *       u^{n+1} = [dt² L u^n + 2m u^n - (m-σ) u^{n-1}] / (m+σ)
 *       then u^{n+1}(node) += wgt·dt²·s_j(t_n)/m(node) over the 2^D multilinear
 *       corners of every source j, and rec_k(t_{n+1}) = Σ wgt·u^{n+1}(node).
 *   Time levels rotate by pointer (§3.3.2: t0 = time mod 2, t1 = (time+1) mod 2).
 *
 * Arrays crossing this boundary are float32, dense, C order, interior only
 * (no halo): 3-D [n0][n1][n2], 2-D [n0][n1], last axis contiguous.  Axis d has
 * shape[d] nodes at coordinates i·spacing[d], i = 0..shape[d]-1.  Coordinates
 * are float32 [npoints][ndim] in the same axis order.  Multilinear corners:
 * x = c/h, i = floor(x), f = x - i, a point on the last node uses i = n-2,
 * f = 1; x within 1e-9·(n-1) beyond an end is snapped onto it; further out is
 * FD_EINVAL.
 *
 * Ownership: every pointer argument is borrowed for the duration of the call;
 * its contents are copied.  By default pointers are host pointers (any host
 * memory; pinned memory makes the copies asynchronous).  With
 * fd_options.device_ptrs = 1 they are device pointers valid on the context's
 * stream.  All library memory is allocated by fd_create/fd_set_* and freed by
 * fd_destroy.
 *
 * Errors: every call returns an fd_status; fd_last_error() gives the text.  A
 * CUDA error makes the context failed: every later call returns FD_ECUDA until
 * fd_destroy.  Calls in the wrong order return FD_ESTATE.  Not thread-safe per
 * context; separate contexts are independent.
 */
#ifndef FD_B300_FD_H
#define FD_B300_FD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fd_ctx fd_ctx; /* opaque, owned by the library */

typedef enum {
  FD_OK = 0,
  FD_EINVAL = 1,       /* bad argument (shape, order, dt above the stability limit, ...) */
  FD_ENOMEM = 2,       /* device or host allocation failed */
  FD_ECUDA = 3,        /* CUDA error; the context is failed from now on */
  FD_ESTATE = 4,       /* call out of order (e.g. fd_run before fd_set_model) */
  FD_ETIMEOUT = 5,     /* a kernel's bounded wait expired (reported by fd_read) */
  FD_EUNSUPPORTED = 6  /* valid request the library does not provide */
} fd_status;

typedef enum { FD_DIFFUSION = 0, FD_ACOUSTIC = 1 } fd_equation;

typedef enum {
  FD_KERNEL_AUTO = 0,  /* 3-D: the pipelined kernel where it applies, else plain;
                          2-D: the row-streaming kernel for diffusion from 4 M points,
                          else plain (fastest on L2-resident grids) */
  FD_KERNEL_PLAIN = 1, /* one thread per point, neighbours through L1/L2 */
  FD_KERNEL_TMA = 2    /* 3-D: TMA-fed shared-memory plane ring, z streamed in registers;
                          2-D: rows staged in shared memory with cp.async, y streamed in
                          registers (bitwise the plain kernel) */
} fd_kernel;

/*
 * Values outside the grid.  FD_BOUNDARY_ZERO: the zero halo (every equation).
 * FD_BOUNDARY_ODD (FD_DIFFUSION only): before each step the halo takes the
 * negated mirror image of the interior about the boundary nodes, u(-k) =
 * -u(k) and u(n-1+k) = -u(n-1-k) along each axis, so every sine mode
 * Π sin(k_d π x_d) is an exact eigenvector of the interior update at every
 * space order (the closed-form decay of §5.1.2's problem then holds beyond
 * so = 2).  Needs n_d - 1 >= space_order/2 on every axis (FD_EINVAL).
 */
typedef enum { FD_BOUNDARY_ZERO = 0, FD_BOUNDARY_ODD = 1 } fd_boundary;

typedef struct {
  double nu;          /* diffusion coefficient ν (FD_DIFFUSION only); default 0.5,
                         the benchmark value of §5.1.2 */
  void *cuda_stream;  /* cudaStream_t for all work; NULL: the library creates one */
  int device_ptrs;    /* 1: array arguments are device pointers (see Ownership) */
  int use_graphs;     /* 1 (default): fd_run replays captured CUDA graphs of the step loop */
  int profile;        /* 1: time the stencil launches with CUDA events (fd_profile):
                         each replayed graph chunk as a whole, or, with
                         use_graphs = 0 and in fd_step_fwi, each launch */
  int kernel;         /* fd_kernel; default FD_KERNEL_AUTO */
  int autotune;       /* 1: fd_create runs fd_autotune on the pipelined kernel (its
                         choice is cached per grid shape, space order and equation
                         for the process); 0 (default): the default tile */
  int boundary;       /* fd_boundary; default FD_BOUNDARY_ZERO */
  int dirichlet_interior; /* FD_DIFFUSION: 1 (default) = update the interior nodes and
                         hold the boundary nodes (§2.1.1's `subdomain=grid.interior`, the
                         §5.1.2 benchmark); 0 = update every node, the values outside
                         the grid given by `boundary` (FD_BOUNDARY_ZERO only) */
} fd_options;

/* Fill *opt with the defaults above.  (Library service; no counterpart in the paper.) */
void fd_options_default(fd_options *opt);

/*
 * Paper: §2.1.1 (Grid(shape, extent) and TimeFunction(time_order, space_order)
 * define the problem; op(time=nt, dt=dt) fixes dt) and §5.1.2 (the benchmark
 * problem's grid, order and time step).
 * Create a context.  ndim ∈ {2,3}; shape[d] ≥ 1 (FD_ACOUSTIC: ≥ 2);
 * spacing[d] > 0; space_order even in [2,16]; dt > 0.  FD_DIFFUSION checks
 * stability here: ν dt Σ_d S/h_d² ≤ 2 with S = -(w_0 + 2 Σ_k (-1)^k w_k);
 * FD_ACOUSTIC checks it in fd_set_model.  Fields start at zero.  opt may be
 * NULL (defaults).  On failure *out is NULL.
 */
fd_status fd_create(fd_ctx **out, int ndim, const int64_t *shape,
                    const double *spacing, int space_order, double dt,
                    fd_equation eq, const fd_options *opt);

/*
 * Paper: §6.2.1 (the seismic acoustic operator, whose model is the squared
 * slowness m and an absorbing damping term).
 * FD_ACOUSTIC: squared slowness m (> 0 everywhere) and damping coefficient
 * damp (≥ 0; NULL means 0).  Rejects dt above the leapfrog limit
 * 2 / sqrt(max(1/m) · Σ_d S/h_d²) with FD_EINVAL.  May be called again,
 * also while steps are in flight: with host pointers the upload runs on a copy
 * stream of the context and overlaps them; the new coefficients are computed on
 * the context stream after them (steps already queued keep the old ones).
 * Returns once they are computed and checked.
 */
fd_status fd_set_model(fd_ctx *ctx, const float *m, const float *damp);

/*
 * Paper: §2.1.1 (initial data written into u.data[0] before the operator runs)
 * and §5.1.2 (the benchmark's initial condition).
 * Set the current time level(s).  FD_ACOUSTIC: u_cur = u^n, u_prev = u^{n-1}
 * (NULL: equal to u_cur).  FD_DIFFUSION: u_cur only (u_prev ignored); the
 * boundary values given here are held (with dirichlet_interior = 1).  Does not change the step counter.
 * With u_prev NULL (or equal to u_cur) the field is uploaded once for both levels.
 */
fd_status fd_set_field(fd_ctx *ctx, const float *u_cur, const float *u_prev);

/*
 * (Library service for repeated shots; no counterpart in the paper.)
 * Start over from rest without uploading a field: u^n = u^{n-1} = 0 on every
 * node (boundary values 0 for FD_DIFFUSION), step counter 0, recorded traces
 * cleared (the next fd_run records row 0 afresh).  Model, sources, receivers
 * and the tile configuration stay.  Asynchronous on the context stream.
 */
fd_status fd_reset(fd_ctx *ctx);

/*
 * Paper: §6.2.1 (point sources injected into the wavefield: the sparse
 * operation the OPS backend could not offload) and §2.1.1 (sparse functions).
 * FD_ACOUSTIC: nsrc point sources at coords [nsrc][ndim] with wavelets
 * [nt][nsrc] (row n = s(t_n) for global step n).  Replaces earlier sources;
 * nsrc = 0 removes them.  fd_run fails with FD_EINVAL if it would pass step nt.
 * With the same nsrc and nt as before, the device buffers are refilled in place
 * and the captured step graphs are kept (an acquisition's next shot).
 */
fd_status fd_set_sources(fd_ctx *ctx, int nsrc, const float *coords, int nt,
                         const float *wavelets);

/*
 * Paper: §6.2.1 (receivers interpolating the wavefield) and §2.1.1 (sparse
 * functions).
 * FD_ACOUSTIC: nrec receivers at coords [nrec][ndim].  Traces are recorded
 * for every step run afterwards: row 0 = interpolation of u at step 0, row
 * n+1 after step n (the library grows the trace buffer as needed).
 * Replaces earlier receivers and clears recorded traces; with the same nrec
 * as before the device buffers (and the captured step graphs) are kept.
 */
fd_status fd_set_receivers(fd_ctx *ctx, int nrec, const float *coords);

/* Paper: §2.1.1 (op(time=nt, dt=dt) applies the update nt times) and §3.3.3
 * (one parallel loop per time step, levels t0/t1 rotating).
 * Advance nt ≥ 0 steps (asynchronous on the context stream). */
fd_status fd_run(fd_ctx *ctx, int nt);

/*
 * Paper: §2.1.1 (the solution is read from u.data after the operator ran).
 * Copy results out and synchronise the stream.  u: current level u^n
 * (dense, interior), NULL to skip.  rec: traces [n+1][nrec] for the steps
 * run so far (n = fd_steps_done), NULL to skip.  Returns FD_ETIMEOUT if a
 * kernel reported an expired wait.
 */
fd_status fd_read(fd_ctx *ctx, float *u, float *rec);

/* Previous level u^{n-1} (FD_ACOUSTIC), for checkpoint/resume; syncs.  (Library
 * service; the paper has no counterpart.) */
fd_status fd_read_prev(fd_ctx *ctx, float *u_prev);

/* (Library service; no counterpart in the paper.)
 * Set the global step counter (resume from a checkpoint at step n ≥ 0).
 * Trace rows 0..n keep their contents (zero in a context that has not run);
 * n = 0 makes the next fd_run record row 0 afresh. */
fd_status fd_set_step(fd_ctx *ctx, int64_t n);

/* Steps advanced so far (the global step counter); -1 for NULL. */
int64_t fd_steps_done(const fd_ctx *ctx);

/*
 * Paper: §5.1.3-§5.1.4 (timed runs of the operator and their roofline).
 * Profiling (fd_options.profile = 1): number of stencil launches timed and
 * their summed CUDA-event time in ms since the last call (a graph chunk's time
 * covers its launches and the gaps between them); synchronises and resets.
 */
fd_status fd_profile(fd_ctx *ctx, int64_t *launches, double *stencil_ms);

/*
 * (No counterpart in the paper: inversion built on the §6.2.1 operator.)
 * Full-waveform-inversion support (gradient of a shot's misfit with
 * respect to m for the §6.2.1 operator).  Device fields in the library's padded layout:
 * fd_field_elems floats each (zero halo included), device pointers.
 *
 * fd_snapshot: copy the current level u^n and the previous level u^{n-1} of
 *   ctx into dst_cur / dst_prev (either may be NULL); asynchronous on the
 *   context stream.  A checkpoint of the forward wavefield.
 * fd_restore: copy them back (step counter unchanged: use fd_set_step).
 * fd_imaging: imaging condition of the adjoint-state gradient,
 *     g[i] += scale · ν(i) · (u_next(i) − 2 u_cur(i) + u_prev(i))
 *   over the interior points, where ν is the current level of the adjoint
 *   context adj and u_next/u_cur/u_prev are snapshots (padded) of the forward
 *   context at steps n+1, n, n-1; g is dense [n0][n1][n2] float32 on the
 *   device.  With adj stepping the adjoint recursion (the forward scheme run
 *   backwards with the receiver residuals injected), scale = -1/dt² gives
 *   dJ/dm for J = ½||traces - d_obs||² where damp = 0 at the sources and
 *   receivers.
 */
int64_t fd_field_elems(const fd_ctx *ctx);
fd_status fd_snapshot(fd_ctx *ctx, float *dst_cur, float *dst_prev);
fd_status fd_restore(fd_ctx *ctx, const float *src_cur, const float *src_prev);
fd_status fd_imaging(fd_ctx *adj, float *g, const float *u_next, const float *u_cur,
                     const float *u_prev, double scale);

/*
 * The same FWI operations fused into a time step of the pipelined kernel (3-D
 * FD_ACOUSTIC; FD_EUNSUPPORTED otherwise), so that the
 * backward sweep neither copies the recomputed wavefield nor re-reads ν:
 *
 * fd_step_fwi: advance ctx one step exactly as fd_run(ctx, 1) does, and in the
 *   stencil's epilogue, at every interior point (padded layout, device,
 *   fd_field_elems floats each):
 *     d2_out (may be NULL):  d2_out = (u^{n+1} − u^n) − (u^n − u^{n−1})
 *     img_g  (may be NULL):  img_g += scale · u^{n+1} · img_d2
 *   with the arithmetic of fd_imaging, so a gradient accumulated this way is
 *   bitwise the one fd_snapshot + fd_imaging give (img_g then padded).
 *   FD_EINVAL if img_g is set without img_d2.  Asynchronous on the stream.
 * fd_field_to_dense: copy the interior of a padded field of ctx into a dense
 *   [n0][n1][n2] device array (asynchronous).
 */
fd_status fd_step_fwi(fd_ctx *ctx, float *d2_out, float *img_g, const float *img_d2,
                      double scale);

/*
 * fd_run_fwi: nt ≥ 0 steps of fd_step_fwi in one call, replayed from captured
 *   CUDA graphs (chunks of up to 64 steps, cached per pointer set): step i uses
 *   d2_out = d2_base + s·stride and img_d2 = img_d2_base + s·stride with s = i,
 *   or s = nt−1−i when reverse = 1 (the adjoint sweep reads a block of second
 *   differences backwards); NULL bases skip that output; img_g as in
 *   fd_step_fwi.  stride (floats) ≥ fd_field_elems when a base is given.
 *   Bitwise the nt single calls.  Asynchronous on the stream.
 * fd_residual: the misfit of ctx's recorded traces against observed data
 *   d_obs [n+1][nrec] (device; n = fd_steps_done): r = traces − d_obs (float),
 *   adj_wav [n][nrec] (device, may be NULL) row j = r row n−j (the adjoint
 *   source wavelet: the residual time reversed, for an adjoint run of n steps),
 *   *J (host, may be NULL; then nothing synchronises) = ½ Σ r² accumulated in
 *   double in a fixed order.  FD_ESTATE without recorded traces.
 */
fd_status fd_run_fwi(fd_ctx *ctx, int nt, float *d2_base, const float *img_d2_base,
                     int64_t stride, int reverse, float *img_g, double scale);
fd_status fd_residual(fd_ctx *ctx, const float *d_obs, float *adj_wav, double *J);
fd_status fd_field_to_dense(fd_ctx *ctx, const float *padded, float *dense);

/*
 * Paper: §2.2 and §2.3.3 (see below).
 * Tile configuration of the pipelined 3-D kernel (FD_KERNEL_TMA/AUTO on 3-D
 * grids).  The paper leaves tiling strategy to the OPS library (§2.2) and
 * cites stencil compilers that block the iteration space per thread to save
 * shared-memory reads (§2.3.3, loop aggregation); here the tile shape and the
 * z-streaming depth are chosen per problem by timing.  Every configuration computes
 * bitwise the same result: a point's update is the same arithmetic whatever
 * tile holds it.
 *
 *   tile_x       points per tile along x: 32 (a lane per point), or 64 (a lane
 *                per pair of adjacent points, 8-byte shared-memory reads; the
 *                same arithmetic per point).  fd_step_fwi and batches run 32:
 *                fd_step_fwi refuses a 64-wide configuration (FD_EUNSUPPORTED)
 *                and fd_batch_add puts the member back to the default
 *   tile_y       points per tile along y: consumer warps × rows per thread,
 *                16 (8 × 2) or 32 (8 × 4); with tile_x 64 from space order 8
 *                also 24 (12 warps × 2 rows: more warps per SM where a
 *                thread's registers allow only one CTA)
 *   zblock       z-streaming depth: consecutive planes a CTA streams on one
 *                tile before it moves to the next (the work is cut into
 *                z-blocks of this height; each cut costs 2R re-read planes)
 *   ctas_per_sm  resident CTAs per SM the persistent grid is sized for
 *   aligned      work split: 0 = every CTA gets an equal run of tile-planes in
 *                z-block-major order (a run may start or end inside a
 *                segment); 1 = CTAs get whole (z-block, tile) segments, at
 *                most one CTA per segment, so that the CTAs holding
 *                neighbouring tiles start their segments together; 2 (tile_x
 *                64 only) = a work queue: z-layers (thick while much work remains, thin at
 *                the end; zblock > 0 caps their height) cut into one item per
 *                tile, taken layer by layer, tile by tile, by whichever CTA is
 *                free, so the items in flight are neighbours at about the same
 *                depth and the CTAs finish together (device memory: 16 bytes
 *                per item, held by the plan).  A new context starts with 1 for
 *                FD_ACOUSTIC, 0 for FD_DIFFUSION
 *   skip_c       FD_ACOUSTIC up to space order 8: 1 = tile-planes where C =
 *                (m−σ)/(m+σ) is 1 at every point (no damping) take C = 1 instead
 *                of loading it (4 of the 20 bytes per point; flags recomputed
 *                after fd_set_model); ignored elsewhere.  New contexts: 0
 *   us_per_step  stencil launch time measured by fd_autotune (µs; 0 when
 *                the configuration was set, not measured)
 *
 * fd_get_tile_config: the configuration fd_run uses; FD_EUNSUPPORTED when the
 *   context runs the plain kernel.
 * fd_set_tile_config: use cfg (tile_x 32 or 0, or 64, tile_y 16, 24 (tile_x 64, space
 *   order ≥ 8) or 32, or 0 for the
 *   default, zblock ≥ 0 with 0 meaning one CTA's share (aligned = 0) or the
 *   height that makes about as many segments as CTAs (aligned = 1) or no cap
 *   on the layer height (aligned = 2), ctas_per_sm ≥ 0 with 0 meaning as many
 *   as fit, aligned 0, 1 or 2, skip_c 0 or 1);
 *   FD_EINVAL for anything else, leaving the current configuration in
 *   place.  Captured graphs are dropped.
 * fd_autotune: time every configuration of the search space (tile_x in {32, 64}
 *   (32 only for fd_autotune_fwi) × tile_y in
 *   {16, 24, 32} × ctas_per_sm in 1..fit × (aligned 0 with zblock in {share/2,
 *   share, 2·share} | aligned 1 with m or 2m z-blocks, m = CTAs / tiles |
 *   aligned 2 with uncapped layers for tile_x 64)
 *   × skip_c {0, 1} where it applies (once a model is set),
 *   reps ≥ 1 launches captured in a CUDA graph and replayed three times
 *   after two warm-up launches (eager batches where the stream cannot capture),
 *   the median replay per launch),
 *   then use the fastest.  The candidate launches step on two scratch
 *   levels copied from the current ones, rotating them as fd_run does, so
 *   the solution is not disturbed; sources are not injected during the trials.  Synchronises the
 *   context stream.  tried (may be NULL) receives up to max_tried measured
 *   configurations, *ntried (may be NULL) how many were measured (which may
 *   exceed max_tried); best (may be NULL)
 *   the chosen one.  FD_ENOMEM when the scratch levels do not fit.
 */
typedef struct {
  int tile_x;
  int tile_y;
  int zblock;
  int ctas_per_sm;
  int aligned;
  int skip_c;
  double us_per_step;
} fd_tile_config;

fd_status fd_get_tile_config(const fd_ctx *ctx, fd_tile_config *cfg);
fd_status fd_set_tile_config(fd_ctx *ctx, const fd_tile_config *cfg);
fd_status fd_autotune(fd_ctx *ctx, int reps, fd_tile_config *best, fd_tile_config *tried,
                      int max_tried, int *ntried);
/*
 * fd_autotune_fwi: the same search for the FWI sweep (FD_ACOUSTIC, pipelined
 * kernel): a candidate's time is one plain step plus one fd_step_fwi step
 * writing the second difference plus one accumulating the imaging condition
 * (two more scratch fields), the kernels of one backward step; configurations
 * without an FWI instance that fits the grid are skipped.  Cached separately
 * from fd_autotune's choice.
 */
fd_status fd_autotune_fwi(fd_ctx *ctx, int reps, fd_tile_config *best, fd_tile_config *tried,
                          int max_tried, int *ntried);

/* (Library service.)  Name of the stencil kernel variant fd_run launches (static string):
 * "stencil3d_tma_<equation>" (32-wide tiles), "stencil3d_xp_<equation>"
 * (64-wide tiles, two x points a lane), "stencil3d_plain", "stencil2d_plain",
 * "stencil2d_stream" (2-D rows staged and streamed) or "stencil2d_stream2" (2-D
 * diffusion at space order 2 or 4 with the zero halo: two steps a launch, u^{n+2}
 * from u^n, bitwise two single steps; a chunk of odd length ends with one single step;
 * the second level then holds an older state, so only fd_read's level is u^n). */
const char *fd_kernel_name(const fd_ctx *ctx);

/*
 * (Library service.)
 * Tile-planes of the current tile configuration whose C tile the pipelined
 * kernel skips (fd_tile_config.skip_c = 1: C = 1 on the whole tile-plane):
 * *flagged of *total.  Both 0 when skip_c is off, no model is set or the plain
 * kernel runs.  Synchronises the context stream.
 */
fd_status fd_skip_c_planes(fd_ctx *ctx, int64_t *flagged, int64_t *total);

/* (Library service.)  CUDA kernels this context has launched so far (kernel nodes of replayed
 * graphs included); -1 for NULL. */
int64_t fd_kernel_launches(const fd_ctx *ctx);

/*
 * z-slab sub-domains: one 3-D FD_ACOUSTIC grid split along axis 0 into slabs,
 * each an ordinary context over its own planes, stepped in lockstep with an
 * R-plane halo exchange after every step (the distributed-memory partitioning
 * of a structured block that the paper's OPS backend leaves to its library,
 * §2.2).  Results are bitwise those of the whole grid: a point's update reads
 * the same values, a source corner is injected by the slab that holds its node
 * (in the same order), and a receiver's trace is the sum of the slabs' partial
 * sums over the corners each holds, which the receiver kernel's reduction order
 * (the two halves along axis 0 added last) makes exactly the whole-grid sum.
 *
 * fd_set_subdomain: ctx (3-D FD_ACOUSTIC, shape[0] planes) holds global planes
 *   [z_origin, z_origin + shape[0]) of a grid with z_global planes.  Source and
 *   receiver coordinates are then global (validated against the global extent);
 *   corners in other slabs are left to them, and the traces fd_read returns are
 *   this slab's partial sums.  Call before fd_set_sources / fd_set_receivers
 *   (FD_ESTATE otherwise); (0, 0) makes the context whole again.  m, damp and
 *   fields given to the context are its own planes only.  Batches refuse
 *   sub-domain contexts.  FD_EUNSUPPORTED for other equations and 2-D.
 * fd_halo_elems: floats in one exchanged face, R · (padded plane); -1 for 2-D.
 * fd_halo_copy: copy src's boundary planes of its current level into dst's own
 *   halo of its current level: side 0 = dst's halo below its first plane from
 *   src's last R planes (src is the slab below), side 1 = dst's halo above its
 *   last plane from src's first R planes.  Ordered after src's queued work and
 *   before src's later work when the contexts have different streams; a peer
 *   copy when they live on different devices.  Both slabs need ≥ R planes.
 * fd_halo_export / fd_halo_import: the same faces through a caller buffer of
 *   fd_halo_elems floats (device pointer), for exchanges the caller carries
 *   between processes (e.g. NCCL send/recv): export side 0 = the first R planes,
 *   1 = the last R; import side 0 = the halo below, 1 = the halo above.
 *   Asynchronous on the context stream.
 * fd_run_slabs: advance every slab (slabs[0] at z = 0 upwards, contiguous,
 *   covering the grid) nt steps: exchange halos, then per step run each slab
 *   one step (fd_run) and exchange.  FD_EINVAL if the slabs do not tile the grid,
 *   FD_ESTATE if they are at different steps.
 * fd_accumulate_traces: acc += this context's recorded traces (device pointer,
 *   [steps+1][nrec] floats), on the context stream: adding every slab's partial
 *   traces into a zeroed buffer, slab by slab, gives the whole grid's traces.
 */
fd_status fd_set_subdomain(fd_ctx *ctx, int64_t z_origin, int64_t z_global);
int64_t fd_halo_elems(const fd_ctx *ctx);
fd_status fd_halo_copy(fd_ctx *dst, int side, fd_ctx *src);
fd_status fd_halo_export(fd_ctx *ctx, int side, float *dst);
fd_status fd_halo_import(fd_ctx *ctx, int side, const float *src);
fd_status fd_run_slabs(fd_ctx *const *slabs, int nslabs, int nt);
fd_status fd_accumulate_traces(fd_ctx *ctx, float *acc);

/* Release everything.  NULL is a no-op. */
void fd_destroy(fd_ctx *ctx);

/*
 * (No counterpart in the paper: serving built on the §6.2.1 operator.)
 * Batches: many FD_ACOUSTIC shots of one space order stepped together, as a
 * serving loop that admits and retires shots between runs needs (continuous
 * batching, built on the §6.2.1 operator).
 * A batch tick advances every member one step with one persistent pipelined
 * kernel for all 3-D members (their tile-planes shared out over the CTAs), one
 * kernel for all 2-D members, one source-injection kernel for the 2-D members
 * (3-D injection is fused) and one receiver kernel for all.  Members stay
 * ordinary contexts: after fd_batch_run, fd_read / fd_run work on them as
 * usual, and a member's results are bitwise those of running it alone.
 *
 * fd_batch_create: cuda_stream = cudaStream_t for the batch's work (NULL: own
 *   stream).  Members on other streams are ordered before and after each run
 *   with events.
 * fd_batch_add: ctx must be FD_ACOUSTIC, of the batch's space order, with a
 *   model set, on the batch's device; 3-D members need the pipelined kernel
 *   and must share their grid spacing (their weights are one kernel
 *   parameter); FD_EUNSUPPORTED otherwise.  The batch borrows
 *   the context: remove it before fd_destroy.  The batched kernel runs the
 *   default tile, so fd_batch_run puts a 3-D member with another tile height
 *   back to the default configuration (fd_set_tile_config) before its tick.
 * fd_batch_run: nticks ≥ 0 steps of every member (FD_EINVAL if a member would
 *   pass its wavelet); asynchronous on the batch stream.
 * fd_batch_remove: drops the member (no wait: its stream already waits for
 *   the batch's last run).
 */
typedef struct fd_batch fd_batch;
fd_status fd_batch_create(fd_batch **out, int space_order, void *cuda_stream);
fd_status fd_batch_add(fd_batch *b, fd_ctx *ctx);
fd_status fd_batch_remove(fd_batch *b, fd_ctx *ctx);
fd_status fd_batch_run(fd_batch *b, int nticks);
int fd_batch_size(const fd_batch *b);
int64_t fd_batch_kernel_launches(const fd_batch *b);
const char *fd_batch_last_error(const fd_batch *b);
void fd_batch_destroy(fd_batch *b);

/*
 * (No counterpart in the paper: the admission measure of serving.)
 * Device bytes fd_create + fd_set_* + fd_run allocate for an FD_ACOUSTIC shot
 * (fields with halo, coefficients, m, staging, traces for nt steps, sparse
 * tables) -- the admission measure of a serving loop.  -1 for bad arguments.
 */
int64_t fd_footprint_bytes(int ndim, const int64_t *shape, int space_order, int nrec, int nt,
                           int nsrc);

/* (Library service.)  Text of the last error on ctx (or of the last failed fd_create when ctx is NULL). */
const char *fd_last_error(const fd_ctx *ctx);

/*
 * Paper: §2.1.1 (u.dx2 at space order so: the central second-derivative
 * stencil whose weights these are) and §5.1.5 (the coefficients computed once,
 * outside the kernel).
 * Host-only helpers (no GPU needed).
 * fd_weights: w_0..w_r (r = space_order/2) of the central second-derivative
 *   stencil, as the library uses them; returns FD_EINVAL for a bad order.
 * fd_stability_symbol: S = -(w_0 + 2 Σ_k (-1)^k w_k) for that order (NaN if bad).
 */
fd_status fd_weights(int space_order, double *w);
double fd_stability_symbol(int space_order);

/* Library version string.  (Library service.) */
const char *fd_version(void);

/*
 * (No counterpart in the paper: failure detection of the pipelined kernel.)
 * Failure-detection self-test: launch a kernel that waits, with the same
 * bounded-wait routine the pipelined stencil uses on its mbarriers, on a
 * barrier phase that nothing completes, with a budget of budget_ms (0, 10000]
 * (converted with the SM clock rate).  *expired = 1 when the wait gave up as it
 * must; *waited_ms (may be NULL) = how long it waited.  Faults nothing.
 */
fd_status fd_selftest_bounded_wait(double budget_ms, int *expired, double *waited_ms);

/*
 * No-allocation acoustic run (the paper has no counterpart; this is a service
 * entry point of the library).
 *
 * For callers that cannot allocate GPU memory: applications whose own memory
 * pool already holds the device (cudaMalloc would fail or would break their
 * accounting), and latency-critical loops where cudaMalloc/cudaFree would stall
 * on device-wide synchronisation.  It advances nt ≥ 0 FD_ACOUSTIC steps (no
 * sources or receivers) with the same arithmetic as fd_run, and allocates
 * nothing: its working copies (two zero-halo time levels, the coefficient
 * fields A and C, the set-up reduction words) live in one file-scope device
 * array of FD_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds
 * until the process exits.
 *
 * Arguments: ndim, shape, spacing, space_order, dt as for fd_create; m (> 0),
 * damp (≥ 0, NULL = 0), u_cur = u^n, u_prev = u^{n-1} (NULL = u_cur) are DEVICE
 * pointers to dense interior arrays; outputs u_out = u^{n+nt} and u_prev_out =
 * u^{n+nt-1} (NULL to skip) are DEVICE pointers the caller owns.  cuda_stream is
 * a cudaStream_t (NULL = legacy default stream); the work is ordered on it.
 *
 * Limits and behaviour:
 *  - the four padded fields must fit: 4 × (n0+2r)(n1+2r)(32 + roundup32(n2+r))
 *    × 4 B + 256 B ≤ FD_NOALLOC_SCRATCH_BYTES (3-D; 2-D has no halo along axis
 *    0), e.g. up to 80³ at space order 8; larger grids return FD_EINVAL with the
 *    byte counts in fd_last_error(NULL).
 *  - the first call on a device looks up the array's device address for that
 *    device (with the device current); make that first call before any stream
 *    capture on that device.
 *  - the call synchronises the stream once, after the coefficient set-up, to
 *    validate m, damp and dt (FD_EINVAL as in fd_set_model); the steps and the
 *    copies into u_out/u_prev_out are then queued on the stream and complete
 *    in stream order.
 *  - every call shares the one array and it keeps the last call's contents:
 *    the call clears what must start at zero itself, but calls whose work
 *    overlaps on the GPU (different streams or host threads without ordering)
 *    race with each other and must not be issued.
 *  - errors: FD_EINVAL / FD_ECUDA / FD_EUNSUPPORTED, text in fd_last_error(NULL).
 */
#define FD_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)
fd_status fd_acoustic_run_noalloc(int ndim, const int64_t *shape, const double *spacing,
                                  int space_order, double dt, const float *m,
                                  const float *damp, const float *u_cur, const float *u_prev,
                                  int nt, float *u_out, float *u_prev_out, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* FD_B300_FD_H */
