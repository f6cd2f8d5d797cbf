/*
 * j2d5pt.h -- C ABI of the GB300 library for the 2D Jacobi 5-point iterative
 * stencil (j2d5pt) with deep temporal blocking.
 *
 * The operation (Zhang et al., "Exploiting Scratchpad Memory for Deep Temporal
 * Blocking", GPGPU'23, Section 3.1, Listing 1): for every interior cell
 *     out[y][x] = W*in[y][x-1] + E*in[y][x+1] + S*in[y-1][x] + C*in[y][x] + N*in[y+1][x]
 * out of place (Jacobi), iterated for a number of time steps.  The paper moves
 * the time loop inside the kernel and keeps tiles on chip for several steps
 * (Sections 3.1 and 3.3, Figure 1); the result does not depend on how the
 * steps are blocked.  The boundary is a one-cell Dirichlet ring held constant
 * (the paper is silent on boundaries).
 *
 * Array layout ("plan layout").  A grid has nx*ny interior cells plus the
 * ring: logical cells (y, x) with 0 <= y <= ny+1 and 0 <= x <= nx+1; row 0,
 * row ny+1, column 0 and column nx+1 are the ring.  Cell (y, x) lives at element
 *     y * pitch + offset + x
 * of a device buffer of (ny+2) * pitch elements, where pitch and offset come
 * from j2d5pt_layout().  The offset puts interior column 1 on a 16-byte
 * boundary; pitch * sizeof(element) is a multiple of 16.  Elements outside the
 * logical array (the `offset` leading elements of each row and the tail
 * padding) are never read; the library may overwrite them in output arrays.
 * Buffers must be 16-byte aligned (cudaMalloc gives 256).  Inputs must be
 * finite.
 *
 * Ownership.  All data buffers are owned by the caller; the library never
 * frees them.  A plan owns its device workspace, freed by
 * j2d5pt_plan_destroy().  Plans are not thread safe; use one plan per thread.
 *
 * Streams and errors.  Run calls are asynchronous on the given CUDA stream
 * (a cudaStream_t passed as void*, NULL = legacy default stream); argument
 * errors are returned synchronously and nothing is enqueued.  Device-side
 * errors (a wait that timed out, a failed bound check) are recorded in the
 * plan and reported by j2d5pt_sync_status(), which synchronises the stream of
 * the last run.  j2d5pt_last_error() gives a message for the most recent
 * failure on the calling thread.
 */
#ifndef J2D5PT_H
#define J2D5PT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct j2d5pt_plan_s *j2d5pt_plan_t;

typedef enum { J2D_F64 = 0, J2D_F32 = 1 } j2d_dtype;

typedef enum {
  J2D_OK = 0,
  J2D_ERR_ARG = 1,         /* invalid argument (null pointer, size, step count) */
  J2D_ERR_ALIGN = 2,       /* buffer not 16-byte aligned */
  J2D_ERR_NOMEM = 3,       /* workspace allocation failed */
  J2D_ERR_DEVICE = 4,      /* CUDA runtime error */
  J2D_ERR_UNSUPPORTED = 5, /* configuration not available on this device */
  J2D_ERR_TIMEOUT = 6,     /* a device-side wait gave up; results are invalid */
  J2D_ERR_BOUNDS = 7       /* a device-side bound check failed */
} j2d_status;

/* Kernel families a plan can run.  AUTO uses the plan's tuned or heuristic choice. */
typedef enum {
  J2D_ALGO_AUTO = 0,
  J2D_ALGO_ONESTEP = 1,  /* one launch per time step, streaming through HBM */
  J2D_ALGO_RESIDENT = 2, /* whole grid held on chip for all steps; one persistent launch.  On a
                            batch: the grids in waves, each wave's grids on chip together for all
                            steps (every grid must fit on chip by itself) */
  J2D_ALGO_BANDS = 3,    /* GPU-wide bands of the grid, processed serially, k steps per visit */
  J2D_ALGO_TILES = 4,    /* independent per-CTA tiles with a k-deep overlapped halo */
  J2D_ALGO_SKEWED = 5,   /* serial tiles in skewed order: each CTA advances a run of rows of a
                            column band tile after tile, k steps per visit, each tile taking its
                            top halo at every step from the tile before it (no overlapped halo
                            in y; the k-deep overlap stays in x).  Forward runs only (adjoint
                            runs of a plan set to it take TILES). */
  J2D_ALGO_STREAM = 6    /* temporal blocking in the register file: each warp sweeps a column
                            band (32 16-byte vectors wide, overlapped halo in x) down a run of
                            rows, advancing k steps per pass as a pipeline held in registers
                            (step t of row i-t as row i arrives); one launch per pass, no shared
                            memory.  k in {4, 6, 8, 10, 12} for FP32, {2, 3, 4, 6} for FP64
                            (J2D_ERR_ARG otherwise; default 8 and 2); box plans: {4, 6, 8} for
                            FP32, {2, 3, 4} for FP64 (default 8 and 2).  Forward runs of single
                            grids only (adjoint runs and batches take TILES).  AUTO takes it for
                            FP32 grids too large for the chip and FP64 grids of 8192^2 cells or
                            more. */
} j2d_algo;

/* Plan options (j2d5pt_set_option / j2d5pt_get_option). */
typedef enum {
  J2D_OPT_ALGO = 0,       /* j2d_algo */
  J2D_OPT_DEPTH = 1,      /* temporal depth k (steps per on-chip visit) for BANDS / TILES / SKEWED */
  J2D_OPT_TILE_WX = 2,    /* TILES / SKEWED: warp strips across a CTA tile (16 / WX down) */
  J2D_OPT_CTAS = 3,       /* persistent grid size (0 = one CTA per SM) */
  J2D_OPT_TIMEOUT_MS = 4, /* device-side wait limit in milliseconds (default 2000) */
  J2D_OPT_VERBOSE = 5,    /* 1 = print the chosen configuration to stderr at run time */
  J2D_OPT_GRAPH = 6,      /* 1 = forward runs are captured into a CUDA graph on first use (per
                             buffers and step count) and replayed by later identical calls */
  J2D_OPT_TIMING = 7,     /* 1 = runs record CUDA events around their stencil kernels, read
                             by j2d5pt_kernel_time (ignored for graph replays) */
  J2D_OPT_FAULT_INJECT = 8, /* testing: 1 = in the resident and bands kernels, one strip with a
                               neighbour in another CTA never publishes its step counter to other
                               CTAs, so that neighbour's bounded waits expire and the run reports
                               J2D_ERR_TIMEOUT */
  J2D_OPT_INT_PATH = 9,     /* FP64: 1 (default) = the cells j2d5pt_arith_info selects are
                               evaluated on the integer pipes; 0 = every cell takes the FMA
                               chain on the FP64 pipe.  Ignored for FP32. */
  J2D_OPT_SWEEP_STEPS = 10  /* TILES, FP32 forward: time steps per sweep of a strip, 2 (default:
                               each exchange of halos carries two steps, the strip reading two
                               cells deep around it) or 1.  Results are identical either way;
                               ignored elsewhere. */
} j2d_option;

/* ---- plans ------------------------------------------------------------- */

/* Plan for one grid of nx*ny interior cells.  weights = {W, E, S, C, N} (host,
 * FP64; rounded to float for J2D_F32 plans; used as given, not normalised).
 * Queries the current CUDA device and allocates the plan's workspace on it. */
j2d_status j2d5pt_plan(j2d5pt_plan_t *plan, int nx, int ny, j2d_dtype dtype,
                       const double weights[5]);

/* Plan for `count` independent grids advanced together (one persistent launch).
 * nx[i], ny[i]: interior sizes; weights: count*5 values, grid i at weights+5*i. */
j2d_status j2d5pt_plan_batched(j2d5pt_plan_t *plan, int count, const int *nx, const int *ny,
                               j2d_dtype dtype, const double *weights);

/* Plan for a second stencil shape through the same kernels: the 3x3 box
 * (j2d9pt), the paper's method applied beyond its j2d5pt case study (title,
 * Section 1; the step function of Section 3.1 does not depend on the shape):
 *     out[y][x] = sum over dy, dx in {-1, 0, 1} of weights[3*(dy+1) + (dx+1)] * in[y+dy][x+dx]
 * i.e. weights row by row from the y-1 row (the row S reads), x-1 first.
 * Same layout, ring and ownership rules as j2d5pt_plan; host FP64 weights
 * (rounded to float for J2D_F32), used as given.  The plan runs forward:
 * j2d5pt_run / j2d5pt_run_host / j2d5pt_autotune and the option, layout,
 * describe, timing and status calls; its algorithms are J2D_ALGO_ONESTEP,
 * J2D_ALGO_SKEWED and J2D_ALGO_STREAM (any other choice runs the skewed
 * tiles; AUTO takes the stream schedule for FP32 grids too large for the
 * chip and FP64 grids of 8192^2 cells or more).  The adjoint,
 * weight-gradient and j2d5pt_set_weights calls return J2D_ERR_UNSUPPORTED.
 * FP64 cells are evaluated as j2d5pt_arith_info describes, with the nine
 * terms: the FMA chain takes the product of the (y-1, x) term, then the
 * (y-1, x-1), (y-1, x+1), (y, x), (y, x-1), (y, x+1), (y+1, x), (y+1, x-1),
 * (y+1, x+1) terms; the integer path the correctly rounded nine-term sum. */
j2d_status j2d9pt_plan(j2d5pt_plan_t *plan, int nx, int ny, j2d_dtype dtype, const double weights[9]);

j2d_status j2d5pt_plan_destroy(j2d5pt_plan_t plan);

/* Replace the weights {W, E, S, C, N} of grid `index` (host, FP64).  Later
 * runs use them; a graph captured under J2D_OPT_GRAPH is discarded. */
j2d_status j2d5pt_set_weights(j2d5pt_plan_t plan, int index, const double weights[5]);

/* Layout of grid `index` (0 for single-grid plans): elements per row and the
 * element offset of logical column 0 (see the layout rules above). */
j2d_status j2d5pt_layout(j2d5pt_plan_t plan, int index, long *pitch, long *offset);

j2d_status j2d5pt_set_option(j2d5pt_plan_t plan, j2d_option opt, long value);
j2d_status j2d5pt_get_option(j2d5pt_plan_t plan, j2d_option opt, long *value);

/* Human-readable description of the configuration the next run will use. */
j2d_status j2d5pt_describe(j2d5pt_plan_t plan, char *buf, size_t len);

/* ---- forward ----------------------------------------------------------- */

/* u_steps = M^steps u_0 (Section 3.1's update applied `steps` times, ring held
 * constant).  in, out: device buffers in plan layout; they may alias.
 * steps = 0 copies.  Asynchronous on `stream`. */
j2d_status j2d5pt_run(j2d5pt_plan_t plan, const void *in, void *out, long steps, void *stream);

/* Same, for a batched plan: in[i], out[i] (host arrays of device pointers) are
 * grid i's buffers in its own layout. */
j2d_status j2d5pt_run_batched(j2d5pt_plan_t plan, const void *const *in, void *const *out,
                              long steps, void *stream);

/* End-to-end form on HOST buffers: h_in and h_out are dense (ny+2) x (nx+2)
 * row-major host arrays (ring included).  Copies in, runs, copies out and
 * synchronises; uses the plan's device workspace.  Pinned host memory gives
 * full copy bandwidth: a pinned h_in is read by a gather kernel on the device
 * (pageable memory takes a plain copy). */
j2d_status j2d5pt_run_host(j2d5pt_plan_t plan, const void *h_in, void *h_out, long steps);

/* Forward run that keeps every intermediate state (the recomputation of a
 * checkpointed gradient): `states` is a device buffer of `steps` consecutive
 * grids in the plan layout, each (ny+2) * pitch elements, 16-byte aligned;
 * state t (1 <= t <= steps, ring included) is written at states + (t-1) *
 * (ny+2) * pitch elements.  Bit-identical to `steps` chained calls of
 * j2d5pt_run(plan, ., ., 1, stream).  With J2D_ALGO_AUTO the one-step
 * kernel runs one launch per state (it writes every state anyway, and
 * measured faster than blocked kernels storing each step); a plan set to a
 * temporally blocked algorithm stores each state from its one persistent
 * launch (the skewed and two-step FP32 schedules run as single-step tiles
 * here); a plan set to J2D_ALGO_STREAM stores every step's rows from its
 * pipeline, one launch per pass of k steps (k in {2, 3, 4} for FP64, {4, 8}
 * for FP32; other depths take 2 and 8).  Single-grid, five-point plans; `in` must not lie
 * inside `states`; steps >= 1.  J2D_ERR_ARG / J2D_ERR_ALIGN /
 * J2D_ERR_UNSUPPORTED as for j2d5pt_run. */
j2d_status j2d5pt_run_states(j2d5pt_plan_t plan, const void *in, void *states, long steps, void *stream);

/* ---- adjoint and gradient (the transpose of the forward map) ------------ */

/* lam_0 = (M^T)^steps lam_T, where M is one forward step over all cells
 * (interior rows of M hold the five weights, ring rows are the identity).
 * Interior cells follow the transposed stencil with weights mirrored
 * (x-1 <- E, x+1 <- W, y-1 <- N, y+1 <- S) and reading only interior cells;
 * ring cells keep their value and add the weight of their link times the
 * adjacent interior value each step; corners are unchanged.  Buffers in plan
 * layout; they may alias. */
j2d_status j2d5pt_run_adjoint(j2d5pt_plan_t plan, const void *lam_T, void *lam_0, long steps,
                              void *stream);

/* dw[d] += sum over interior cells i of lam_t1[i] * u_t[nbr_d(i)], d = W, E, S,
 * C, N (nbr = x-1, x+1, y-1, self, y+1): the gradient contribution of one
 * step t of L = <g, u_T> with lam_t1 = (M^T)^(T-t-1) g.  dw: 5 doubles in
 * device memory, accumulated (not overwritten).  The sum is reduced in a
 * fixed order, so results are reproducible. */
j2d_status j2d5pt_weight_grad(j2d5pt_plan_t plan, const void *u_t, const void *lam_t1,
                              double *dw, void *stream);

/* One backward step of the gradient in one pass: lam_t = one adjoint step of
 * lam_t1 (the same values as j2d5pt_run_adjoint(plan, lam_t1, lam_t, 1)) and
 * dw += the weight_grad contribution of (u_t, lam_t1) (as j2d5pt_weight_grad,
 * reduced in another fixed order, so the sums may differ from it in the last
 * bits).  Single-grid plans; lam_t must not alias lam_t1 or u_t.  Buffers in
 * the plan layout, 16-byte aligned; dw 5 doubles in device memory.
 * Asynchronous on `stream`. */
j2d_status j2d5pt_adjoint_step_wgrad(j2d5pt_plan_t plan, const void *u_t, const void *lam_t1, void *lam_t,
                                     double *dw, void *stream);

/* Same reduction for callers that cannot allocate device memory; no plan
 * needed.  The paper has no counterpart to this call.
 * Callers that cannot call cudaMalloc: code running while a stream is being
 * captured into a CUDA graph, code whose device memory is owned by a
 * framework's caching allocator, and latency-bound loops that cannot absorb
 * cudaFree's device-wide synchronisation.  Allocates nothing: its scratch (the
 * per-block partial sums) is a fixed 2.5 MiB device array inside the library,
 * which every GPU that loads the library holds until the process exits.
 * u_t and lam_t1 are nx*ny grids in the plan layout j2d5pt_plan would give for
 * (nx, ny, dtype); dw as for j2d5pt_weight_grad (accumulated).  Grids needing
 * more than 65536 partial-sum blocks (about 1.1e9 FP64 or 2.1e9 FP32 cells)
 * are rejected with J2D_ERR_ARG.  The first call on each device looks up the
 * array's device address (once, with that device current; again after the
 * device's context was reset); make it before any stream capture.  All calls share the one array: calls that overlap on
 * the GPU (other streams, other threads) race and give wrong results;
 * serialise them.  Asynchronous on `stream`. */
j2d_status j2d5pt_weight_grad_noalloc(int nx, int ny, j2d_dtype dtype, const void *u_t,
                                      const void *lam_t1, double *dw, void *stream);

/* ---- status, tuning, diagnostics ---------------------------------------- */

/* Synchronise the stream of the plan's last run and return its device-side
 * status (J2D_OK, J2D_ERR_TIMEOUT, J2D_ERR_BOUNDS) or a CUDA error; clears it. */
j2d_status j2d5pt_sync_status(j2d5pt_plan_t plan);

/* Time the candidate configurations for `steps` steps on the given buffers
 * (out is overwritten; in is only read unless in == out) and keep the fastest
 * in the plan.  Results are cached in the file named by J2D_TUNE_CACHE if set.
 * Synchronous. */
j2d_status j2d5pt_autotune(j2d5pt_plan_t plan, const void *in, void *out, long steps,
                           void *stream);

/* Same for a batched plan (in[i], out[i] as for j2d5pt_run_batched); picks the
 * temporal depth and tile shape of the batched kernel. */
j2d_status j2d5pt_autotune_batched(j2d5pt_plan_t plan, const void *const *in, void *const *out,
                                   long steps, void *stream);

/* Device time in milliseconds from just before the first to just after the
 * last stencil kernel of the plan's most recent run (ring copies and other
 * set-up excluded), with J2D_OPT_TIMING set.  Synchronises on the end event. */
j2d_status j2d5pt_kernel_time(j2d5pt_plan_t plan, double *ms);

/* Measured fused multiply-add throughput of the current device for `dtype`
 * (FMA instructions per second), from a short dependent-free FMA loop.  Used
 * as the arithmetic roofline. Synchronous. */
j2d_status j2d5pt_measure_fma_rate(j2d_dtype dtype, double *fma_per_s);

/* Measured shared-memory bandwidth of the current device (bytes per second,
 * loads plus stores), from 16-byte lane-consecutive accesses (the pattern of
 * the strip sweeps) on every SM.  The shared-memory roofline of the DTB
 * kernels.  Synchronous. */
j2d_status j2d5pt_measure_smem_bandwidth(double *bytes_per_s);

/* Measured throughput of the FP64 integer path alone (cells per second on
 * the current device; see j2d5pt_arith_info), from a short loop of
 * independent cell evaluations with register inputs.  With the FMA rate this
 * gives the arithmetic roofline of the FP64 kernels.  Synchronous. */
j2d_status j2d5pt_measure_exact_rate(double *cells_per_s);

/* The same for the nine-term integer path of the 3x3 box (cells per second). */
j2d_status j2d9pt_measure_exact_rate(double *cells_per_s);

/* FP64 cell arithmetic (all kernels alike, so results do not depend on the
 * algorithm, depth or tiling).  With J2D_OPT_INT_PATH = 1 (the default), a
 * cell (x, y) for which bit ((y & 3) * 2 + (x & 1)) of *exact_mask is set, and
 * whose five weights and
 * five input values are positive normal numbers with product exponents
 * within *exact_guard bits of each other and a normal result, gets the
 * correctly rounded (nearest-even) value of the exact five-term sum,
 * computed on the integer pipes.  Every other FP64 cell, and every FP32
 * cell, gets the FMA chain r = S*in[y-1][x]; r = fma(C, in[y][x], r);
 * r = fma(W, in[y][x-1], r); r = fma(E, in[y][x+1], r);
 * r = fma(N, in[y+1][x], r) (the adjoint uses its own link weights in the
 * same roles).  Either pointer may be NULL.  Never fails. */
j2d_status j2d5pt_arith_info(unsigned *exact_mask, int *exact_guard);

/* Geometry of the stream schedule (J2D_ALGO_STREAM) for an nx x ny grid of
 * the given dtype and shape (5: five-point, 9: the 3x3 box) at `depth` steps
 * per pass, when the device holds `resident_warps` warps of the stream kernel
 * at once (a plan takes that from the kernel's occupancy and the SM count).
 * Host arithmetic only, no device call.  out[0..5] = {steps per pass k, halo
 * columns G on each side of a band (k rounded up to a whole 16-byte vector),
 * stored columns per band (32 vectors' worth minus 2G), bands
 * (ceil(nx / stored columns)), rows stored per run H, runs per band}: band b
 * stores columns [1 + b*(stored), ...) and run r rows [1 + r*H, ...), each
 * clipped to the grid.  J2D_ERR_ARG for sizes < 1, an unknown dtype or shape,
 * a depth with no stream kernel, resident_warps < 1 or a NULL out. */
j2d_status j2d5pt_stream_geometry(int nx, int ny, j2d_dtype dtype, int shape, int depth, long resident_warps,
                                  long out[6]);

/* Number of CUDA kernels this library has launched in this process so far
 * (all threads, all plans); a diagnostic for launch accounting. */
long j2d5pt_kernel_launches(void);

/* Message for the most recent failing call on this thread ("" if none). */
const char *j2d5pt_last_error(void);

/* Library version string. */
const char *j2d5pt_version(void);

#ifdef __cplusplus
}
#endif

#endif /* J2D5PT_H */
