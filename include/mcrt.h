/*
 * mcrt.h -- C ABI of the GB300 reciprocal Monte Carlo radiative-transfer library.
 *
 * The library computes the radiative source Q_rad [W/m^3] of every cell of a 3D
 * Cartesian channel grid with the emission-based reciprocal Monte Carlo (ERMC)
 * method of Silvestri & Pecnik (arXiv:1810.00188): Section 2 (Eqs. 1-14), the
 * narrow-band correlated-k sampling of Section 2.1 (Eqs. 15-17), and the
 * initialise / march / residual-dump steps of Algorithm 1.  The paper's problem
 * statement (Section 2.2, Algorithm 2) gives the inputs: the grid, the
 * temperature field, the absorption-coefficient and blackbody tables, the number
 * of rays per cell and the transmissivity cut-off; the output is Q_rad per cell.
 *
 * Conventions shared by every call:
 *  - Every call returns an mcrt_status code and never throws or aborts.
 *  - Arrays are plain pointers.  `mem` says whether a pointer is host memory
 *    (MCRT_MEM_HOST) or device memory of the context's GPU (MCRT_MEM_DEVICE).
 *  - Field arrays are [nz][ny][nx] with x fastest: cell (i,j,k) is element
 *    i + nx*(j + ny*k).  y is the wall-normal direction; x and z are periodic.
 *  - set_* calls COPY their inputs into library-owned device memory; the caller
 *    keeps ownership of its pointers and may reuse them when the call returns.
 *  - Output buffers are caller-owned and hold one value per emitting cell of the
 *    solve's box, x fastest within the box.
 *  - `cuda_stream` is a cudaStream_t (NULL: the legacy default stream).  Device
 *    work is ordered on that stream.  With MCRT_MEM_DEVICE outputs the solve is
 *    asynchronous (like the paper's kickoff kernel, Algorithm 2); with
 *    MCRT_MEM_HOST outputs it returns after the results are on the host.
 *  - A context belongs to one thread at a time.  There is no CPU fallback: a
 *    missing or unusable GPU yields MCRT_E_CUDA.
 */
#ifndef MCRT_H
#define MCRT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mcrt_ctx mcrt_ctx; /* opaque, library-owned */

typedef enum {
  MCRT_OK = 0,
  MCRT_E_ARG = 1,         /* NULL pointer, bad size, value out of its domain    */
  MCRT_E_STATE = 2,       /* solve before set_kdist / set_fields                */
  MCRT_E_CUDA = 3,        /* CUDA runtime error (no device, launch failure, ...) */
  MCRT_E_OOM = 4,         /* device allocation failed                           */
  MCRT_E_RANGE = 5,       /* non-finite or non-positive T, negative or NaN x     */
  MCRT_E_TIMEOUT = 6,     /* a bounded device-side wait gave up                 */
  MCRT_E_UNSUPPORTED = 7  /* valid request this build does not implement         */
} mcrt_status;

enum { MCRT_MEM_HOST = 0, MCRT_MEM_DEVICE = 1 };
/* MCRT_FP32: traversal, table lookups, exp, the ray weight (a binary64 host
 * table rounded once) and each ray's sample Y in binary32; the per-cell tallies
 * sum Y and Y^2 in binary64 with Neumaier compensation (runs of 32 samples
 * summed exactly first, the runs added in segments of up to 64 and the segments
 * in order; mcrt_tuning.tally_binary32 selects compensated binary32 pairs
 * instead).  MCRT_FP64: everything binary64. */
enum { MCRT_FP32 = 0, MCRT_FP64 = 1 };
/* Ray origin: uniform in the cell volume (f_V = 1/V_i, Eq. 4) or the cell centre
 * (Algorithm 1, "ray.pos <- cell.center"). */
enum { MCRT_ORIGIN_UNIFORM = 0, MCRT_ORIGIN_CENTER = 1 };
/* Spectral/directional proposal: Zhang's T_max Planck-kappa pdf (Eq. 13,
 * discretised as Eq. 16) with isotropic directions, or per-cell pdfs supplied by
 * mcrt_set_cell_proposal. */
enum { MCRT_PROPOSAL_PLANCK_TMAX = 0, MCRT_PROPOSAL_CELL = 1 };
/* Reciprocal estimator (Section 2, Eq. FM with the reciprocity relation).
 * ERMC: cell i's exchanges from cell i's own rays (Eq. 14 per ray).
 * ARMC: cell i's exchange with every other medium cell from the rays emitted by
 *   that cell and absorbed in i (each ray deposits minus its emission-based
 *   segment term into the absorbing cell, its residual into the last cell it
 *   crossed); its exchange with the walls from its own rays.  The paper notes it
 *   has the lower variance where the gas is cold and absorbs.
 * HYBRID: per cell lam Q_ERMC + (1 - lam) Q_ARMC from the same rays, lam =
 *   (T_i - T_min) / (T_max - T_min) over the medium. */
enum { MCRT_EST_ERMC = 0, MCRT_EST_ARMC = 1, MCRT_EST_HYBRID = 2 };
enum { MCRT_REFLECT_DIFFUSE = 0, MCRT_REFLECT_SPECULAR = 1 };

/* Grid and walls (Section 2.2: finite volumes with index (i,j,k); Eq. 3: the
 * wall emissivity eps_w enters the transmissivity).  Cells of size lx/nx x dy_j
 * x lz/nz: uniform in the periodic x and z; in y uniform (ly/ny) or stretched
 * by a list of faces, like the wall-refined channel DNS grids of Section 5.
 * Wall 0 is y = 0, wall 1 is y = ly.  eps_wall = 1 is a black wall (the ray
 * ends there); 0 <= eps < 1 reflects the rest. */
typedef struct {
  int nx, ny, nz;          /* >= 1 each; nx*ny*nz < 2^31                          */
  double lx, ly, lz;       /* box lengths [m], > 0                                */
  double eps_wall[2];      /* in [0, 1]                                           */
  double T_wall[2];        /* [K], >= 0                                           */
  int reflect;             /* MCRT_REFLECT_*                                      */
  int device;              /* CUDA device ordinal                                 */
  const double *yf;        /* host [ny + 1] wall-normal faces, strictly increasing,
                              yf[0] = 0 and yf[ny] = ly; copied by mcrt_create;
                              NULL: uniform ly / ny                              */
  int xz_walls;            /* 0: x and z periodic (a channel); 1: a closed box
                              with black walls on the x and z faces too (the
                              paper's 3D verification cases 3 and 4, Table 1)   */
  double T_xz[4];          /* [K] of the x = 0, x = lx, z = 0, z = lz walls     */
} mcrt_grid_desc;

/* Narrow-band correlated-k tables (Section 2.1, Eq. 16; Section 2.2: tabulated
 * blackbody intensity and absorption coefficient, linear interpolation in T).
 * T nodes are T0 + t*dT, t = 0..nT-1; temperatures outside are clamped to the
 * end nodes.  kappa(T, x) = kappa_table(T) * x / x_ref. */
typedef struct {
  int n_bands, n_g;        /* n_bands in [1, 1024], n_g in [1, 64]               */
  const double *w_g;       /* [n_g] quadrature weights, >= 0                      */
  double T0, dT;           /* dT > 0                                              */
  int nT;                  /* >= 2                                                */
  const double *kappa;     /* [n_bands][n_g][nT] [1/m] at x_ref, finite, >= 0     */
  const double *B;         /* [n_bands][nT] band intensity [W m^-2 sr^-1], >= 0;
                              NULL: the library computes it from nu_c and dnu   */
  double x_ref;            /* > 0                                                 */
  const double *nu_c;      /* [n_bands] band centres [1/cm], > 0; read only when
                              B is NULL                                          */
  const double *dnu;       /* [n_bands] band widths [1/cm], > 0; read only when
                              B is NULL: B_n(T) = dnu 2 h c^2 nu^3 /
                              (exp(h c nu / (k T)) - 1) at the band centre, with
                              nu = 100 nu_c [1/m] and the exact SI constants;
                              T <= 0 gives 0 (Section 2.2 tabulates the
                              blackbody intensity for the narrow bands)          */
} mcrt_kdist_desc;

typedef struct {
  int rays_per_cell;       /* N_r of Eq. 8, >= 1                                  */
  int max_steps;           /* cap on medium segments per ray (>= 1); a capped ray
                              dumps its residual like the tol cut-off            */
  double tol;              /* transmissivity cut-off of Algorithm 1, in (0, 1)    */
  uint64_t seed;           /* Philox key                                          */
  uint64_t ray_offset;     /* rays use indices ray_offset .. ray_offset+N-1       */
  uint32_t snapshot;       /* fourth Philox counter word                          */
  int precision;           /* MCRT_FP32 or MCRT_FP64                              */
  int origin;              /* MCRT_ORIGIN_*                                       */
  int proposal;            /* MCRT_PROPOSAL_*                                     */
  int use_box;             /* 0: all cells emit; 1: only the box below            */
  int box[6];              /* i0,i1,j0,j1,k0,k1, half-open, may be empty          */
  uint64_t *steps_out;     /* optional per-cell medium-segment counts (same `mem`
                              as the outputs), or NULL                           */
  /* Multigrid (Section 4.3, "Multigrid"): rays march on overlaid grids that
   * coarsen by 2, mg_steps segments on each grid before falling onto the next
   * coarser one at their current point, and run to termination on the
   * coarsest.  Grid l + 1 halves every dimension of grid l and holds the mean T
   * and x of the 2x2x2 cells it covers; it exists while every dimension of
   * grid l is even and halves to at least 3 cells (mcrt_multigrid_levels).
   * An approximation of the single-grid estimate (the coarse cells average T
   * before the table lookups), not an unbiased estimator of it. */
  int mg_levels;           /* grids used, 0 or 1: the grid itself (exact march)   */
  int mg_steps;            /* segments per grid but the coarsest, >= 1 when
                              mg_levels > 1 (the paper uses 5)                   */
  /* MCRT_EST_*.  ARMC and HYBRID: MCRT_FP32 or MCRT_FP64, the whole grid (every
   * cell emits; no box) and one grid, on channel grids (uniform or stretched wall-normal
   * faces; deposits carry the volume ratio of the emitting and the absorbing
   * cell) and closed boxes (the x/z wall terms stay in the emitting cell); long
   * rays are handed to the warp-parallel march, which makes their deposits, as
   * in the emission-based solve; anything else is refused with
   * MCRT_E_UNSUPPORTED.  sigma_out is the batch-means standard error over K =
   * min(16, rays_per_cell) batches of ray indices (r mod 16).  The deposits are
   * binary64 atomic adds, so these results are reproducible to rounding, not bit
   * for bit; p->steps_out and mcrt_get_stats count the cells' own rays. */
  int estimator;
} mcrt_solve_params;

typedef struct {
  uint64_t steps;          /* medium segments marched by the last solve           */
  uint64_t rays;           /* rays traced                                         */
  uint64_t capped;         /* rays stopped by max_steps                           */
  uint64_t wall_hits;      /* wall events                                         */
  uint64_t max_ray_steps;  /* medium segments of the longest ray                  */
  double T_max;            /* temperature of the plain proposal (Eq. 13)          */
  float kernel_ms;         /* device time of the last solve's trace launch        */
  int launches;            /* kernels the last solve launched                     */
  uint64_t long_rays;      /* FP32: rays finished by the warp-parallel march      */
  uint64_t long_overflow;  /* FP32: long rays that found the hand-off buffer full
                              and were finished where they started (see
                              mcrt_tuning); 0 in every solve whose results are
                              bitwise independent of the launch shape            */
  float trace_ms;          /* FP32 solves: device time of the trace kernel alone,
                              the warp-parallel march of the long rays, and the
                              per-cell reduction (CUDA events recorded on the
                              solve's stream between the launches, summed over
                              chunks); 0 for FP64 solves                          */
  float long_ms;
  float reduce_ms;
} mcrt_solve_stats;

/* Launch shape of the FP32 trace kernel.  The paper sizes its launches so that
 * "the GPU resources are fully utilized" (Section 3); here the choice is left to
 * an autotuner.  Q, sigma and the step counts do not depend on the launch shape
 * (CTAs per SM, steps per round, scratch): every cell's samples are reduced in a
 * fixed order.
 *
 * Long rays.  A ray of an optically thin band that runs nearly parallel to the
 * walls crosses up to ~10^5 cells of the periodic directions, one dependent
 * gather after another; the solve cannot end before its last step.  The FP32
 * exact march therefore hands such a ray off: when it has marched
 * long_ray_steps segments (or reflects off a wall after that) and at least
 * long_ray_flight x/z face crossings remain before its next y face, its state
 * moves to a device buffer, and a second kernel finishes it with a whole warp,
 * the 32 lanes marching consecutive pieces of the flight at once and combining
 * them with a product scan of the transmissivities.  The estimate is the same
 * path integral (Eqs. 2, 3, 14) in another summation order.  These two
 * thresholds are part of the estimator's arithmetic: results are bitwise
 * reproducible for fixed thresholds (unless the hand-off buffer overflows,
 * which mcrt_get_stats reports). */
typedef struct {
  int min_blocks_per_sm;   /* 0: default (3); 1..4 CTAs of 256 threads per SM,
                              trading registers per thread against occupancy */
  int steps_per_round;     /* 0: default (1); 1, 2 or 4 march steps per lane
                              between refills of idle lanes                      */
  int scratch_mib;         /* 0: default (4096); cap of the per-ray sample
                              scratch; larger solves run in several chunks      */
  int long_ray_steps;      /* 0: default (1024); > 0: hand-off threshold in
                              segments; < 0: never hand off                     */
  int long_ray_flight;     /* 0: default (32); > 0: x/z crossings left in the
                              flight for a hand-off; < 0: any flight            */
  int tally_binary32;      /* 0 (default): binary64 per-cell tallies -- each run
                              of 32 samples of a cell summed exactly, the runs
                              added with Neumaier's compensated binary64 sum in
                              segments of up to 64 runs, the segments added the
                              same way (within about 2^-51 of sum |Y| of the
                              exact sum of the samples); 1: compensated binary32
                              pairs (within about 2e-7 of sum |Y|), a little
                              cheaper */
  int tally_plain_loads;   /* 0 (default): the binary64 tallies read the samples
                              through the tensor memory accelerator (tiled bulk
                              copies into shared memory) where their layout
                              allows it (rays_per_cell % 4 == 0); 1: by plain
                              loads.  The same results either way.  Batches
                              use plain loads (their launches share the SMs) */
  int claim_rays;          /* 0: default (1024); FP32 solves: rays per run of
                              cells a warp claims at a time (the run is at
                              least one cell and at most 1/8 of a warp's share
                              of the solve); results do not depend on it      */
  int batch_per_snapshot;  /* read from items[0]'s context by mcrt_batch_create:
                              0 (default): a batch whose items share the
                              k-distribution is one persistent launch over all
                              items; 1: per-item launches in `streams` graph
                              branches, as for mixed k-distributions (the same
                              results; which is faster depends on the batch) */
} mcrt_tuning;

/* Number of overlaid grids the multigrid march can use on an nx x ny x nz grid
 * (1 when no dimension pair allows a coarser grid): the paper's counts, e.g.
 * 3 for 16^3, 5 for 64^3, 6 for 128^3, 7 for 192^3 (Sections 4.3 and 5).
 * Returns 0 for a non-positive dimension. */
int mcrt_multigrid_levels(int nx, int ny, int nz);

/* Creates a context on grid->device.  *out receives the handle (NULL on error).
 * Errors: MCRT_E_ARG (bad geometry / walls / faces), MCRT_E_CUDA (no such
 * device). */
int mcrt_create(const mcrt_grid_desc *grid, mcrt_ctx **out);

/* Copies the k-distribution tables (Section 2.1-2.2) to the device and builds
 * the FP32 and FP64 interpolation nodes.  With kd->B NULL, the band intensities
 * on the T nodes are first computed on the host in binary64 from kd->nu_c and
 * kd->dnu (the Planck law at each band centre times its width).  The caller
 * keeps ownership of every array; nothing is retained after the call.
 * Synchronous.  Errors: MCRT_E_ARG (a NULL table, B NULL without nu_c and dnu,
 * sizes out of range, a negative or non-finite entry, a non-positive band
 * centre or width). */
int mcrt_set_kdist(mcrt_ctx *ctx, const mcrt_kdist_desc *kd);

/* Copies the temperature field T [K] and the H2O mole fraction x (NULL: x_ref
 * everywhere) into the context -- the paper's host-to-device copy of T
 * (Algorithm 2).  dtype_is_fp64 selects double (1) or float (0) inputs.
 * Validates the field and finds its maximum temperature (one device reduction
 * and a 32-byte read-back on cuda_stream: the call returns after it).
 * Errors: MCRT_E_ARG, MCRT_E_STATE (x_h2o = NULL before mcrt_set_kdist, which
 * supplies x_ref), MCRT_E_RANGE (NaN/inf or T <= 0, x < 0 or non-finite: the
 * field is rejected and the previous one is forgotten). */
int mcrt_set_fields(mcrt_ctx *ctx, const void *T, const void *x_h2o, int dtype_is_fp64, int mem,
                    void *cuda_stream);

/* Supplies per-emitting-cell proposals for MCRT_PROPOSAL_CELL solves (one per
 * cell of the whole grid): cumulative counts of 2^32 over the bands
 * cn[ncells][n_bands] and over g within each band cg[ncells][n_bands][n_g] (each
 * row non-decreasing, last entry 2^32, a band/g with non-zero kappa must have a
 * non-zero count for the estimate to stay unbiased), and the upward-hemisphere
 * (d_y > 0) count hemi[ncells] of 2^23 in [1, 2^23 - 1].  The ray weight uses
 * these exact probabilities (Eq. 14 with the pdfs of Eqs. 4, 9, 16 replaced).
 * Copies; synchronous.  Errors: MCRT_E_ARG, MCRT_E_STATE (no kdist). */
int mcrt_set_cell_proposal(mcrt_ctx *ctx, const uint64_t *cn, const uint64_t *cg,
                           const uint32_t *hemi, int mem, void *cuda_stream);

/* Estimates Q_rad for every emitting cell of the box: rays_per_cell rays per
 * cell, each drawn with Philox4x32-10 at counter (cell, ray, block, snapshot)
 * and key seed, marched cell by cell until tau <= tol, a black wall, or
 * max_steps, tallying kappa_i (I_b,i - I_b,j) tau alpha_j (Eqs. 2, 3, 14) and the
 * residual dump of Algorithm 1.  q_out[c] = the mean of the per-ray samples
 * (Eq. 8) in W/m^3 (> 0: the cell cools); sigma_out[c] (nullable) = its
 * standard error.  Output pointers are caller-owned, box-sized, `mem` memory.
 * Errors: MCRT_E_ARG, MCRT_E_STATE (no fields or kdist, or no cell proposal for
 * MCRT_PROPOSAL_CELL), MCRT_E_CUDA, MCRT_E_OOM. */
int mcrt_solve_qrad(mcrt_ctx *ctx, const mcrt_solve_params *p, double *q_out, double *sigma_out,
                    int mem, void *cuda_stream);

/* Sets / reads the launch shape used by later FP32 solves.  Errors: MCRT_E_ARG
 * (value out of range). */
int mcrt_set_tuning(mcrt_ctx *ctx, const mcrt_tuning *t);
int mcrt_get_tuning(const mcrt_ctx *ctx, mcrt_tuning *t);

/* Waits for the last solve and reports its counters.  Errors: MCRT_E_STATE (no
 * solve yet), MCRT_E_CUDA. */
int mcrt_get_stats(mcrt_ctx *ctx, mcrt_solve_stats *out);

/* Allocation-free solve.  The paper has no counterpart: this is a service for
 * callers that may not allocate device memory while they run -- hosts that
 * reserve the GPU's memory up front and treat any later cudaMalloc as an error or
 * an unpredictable stall (a DNS code that owns the device between its own time
 * steps, a serving process with a fixed memory plan).  It computes the same
 * estimate as mcrt_solve_qrad with MCRT_FP32 and device outputs, on a context
 * whose k-distribution and fields are already set, but calls no cudaMalloc or
 * cudaFree: its scratch (per-ray samples, per-cell step sums, counters) lives in a
 * static device array of 64 MiB that every GPU that loads the library holds until
 * the process exits.
 *  - q_out, sigma_out (nullable) and p->steps_out (nullable) are device pointers,
 *    box-sized as for mcrt_solve_qrad; the call is asynchronous on cuda_stream.
 *  - The first call on a device looks up the array's device address on that
 *    device (cudaGetSymbolAddress).  Under CUDA's lazy module loading (the
 *    default since CUDA 12.2) that look-up is what loads the array -- a one-time
 *    64 MiB device allocation -- and the first launch of each kernel loads its
 *    code.  So make one call per device during set-up, before the host reserves
 *    its memory and before any stream capture (or run with
 *    CUDA_MODULE_LOADING=EAGER); later calls allocate nothing.
 *  - The first call after mcrt_set_kdist, or after an mcrt_set_fields that
 *    changes the proposal's T_max (the largest of the field's and the emitting
 *    walls' temperatures), rebuilds the plain proposal (Eqs. 13, 16) on the host
 *    from fixed buffers and uploads it from pageable memory (the call returns
 *    once the copies are staged); make that call outside stream capture too.
 *  - 8 MiB of the array holds the long rays handed to the warp-parallel march
 *    (2^16 entries, the least buffer of a regular solve), so the results equal
 *    mcrt_solve_qrad's bit for bit unless more rays than that are handed off.
 *  - Large boxes run in several launches, each holding as many cells' samples as
 *    fit; rays_per_cell above what one cell's samples can hold in the rest of the
 *    array (about 14.6 million) is rejected with MCRT_E_ARG and a message giving
 *    the limit.
 *  - Every call shares the array and leaves the last call's contents in it (the
 *    counters and step sums are cleared at the start of each call); calls whose
 *    work overlaps on the GPU -- on different streams of one device -- race and
 *    corrupt each other's results.
 *  - mcrt_get_stats does not report this call.
 * Errors: as mcrt_solve_qrad, plus MCRT_E_ARG when precision is not MCRT_FP32. */
int mcrt_solve_qrad_noalloc(mcrt_ctx *ctx, const mcrt_solve_params *p, double *q_out,
                            double *sigma_out, void *cuda_stream);

/* Batched snapshots (no counterpart in the paper, which solves one field per
 * call; its DNS coupling solves one snapshot per time step, Section 5).  A batch
 * solves many contexts -- snapshots of possibly different grid sizes, each with
 * its k-distribution and fields set -- in one CUDA-graph launch.
 *  - When every item has the same k-distribution (up to 1024 items), the graph
 *    holds ONE persistent FP32 trace launch over all the items' cells, the
 *    warp-parallel march of the long rays it hands off, and one per-cell
 *    reduction (per scratch chunk: the sample scratch covers the whole batch
 *    when it fits in half the free device memory).  Warps claim runs of
 *    cells of the concatenated snapshots, largest snapshot first; a warp lets
 *    its rays finish before it moves on to another snapshot.  `weights` and
 *    `streams` are not used.  mcrt_tuning.batch_per_snapshot = 1 on items[0]'s
 *    context selects the next form instead.
 *  - Otherwise each item is one persistent FP32 trace kernel (and its per-cell
 *    reduction) inside the graph; `streams` concurrent branches run the items in
 *    decreasing order of `weights` (NULL: cell counts), round-robin.  Without
 *    weights every item's kernel is a full wave of persistent CTAs, so one
 *    kernel's tail overlaps the next one's start; with weights each item gets
 *    that share of one wave (meant for streams = n: all items at once).
 * The solve parameters (FP32 only, whole grids; p->box, p->snapshot,
 * p->ray_offset and p->steps_out are ignored) and the launch shape and
 * long-ray thresholds of items[0].ctx are fixed at creation; the items'
 * contexts should share those thresholds for the next sentence to hold.  Every
 * item's result equals its own
 * mcrt_solve_qrad with the item's snapshot word, bit for bit. */
typedef struct mcrt_batch mcrt_batch;
typedef struct {
  mcrt_ctx *ctx;           /* distinct contexts on one device                    */
  double *q_out;           /* device, the item's whole grid (x fastest)          */
  double *sigma_out;       /* device or NULL                                     */
  uint32_t snapshot;       /* fourth Philox counter word of the item             */
} mcrt_batch_item;

/* Builds the batch: proposals, scratch, and the captured graph.  items[0..n-1]
 * are the snapshots; weights (host, n values > 0, or NULL) their relative cost;
 * streams (>= 1, clamped to n) the number of concurrent graph branches (both
 * only for items with different k-distributions).  There, items of one branch
 * run one after another and share that branch's sample scratch (the largest
 * item's chunk, capped by items[0].ctx's scratch_mib).  Synchronous;
 * allocates.  Errors: MCRT_E_ARG, MCRT_E_STATE, MCRT_E_UNSUPPORTED, MCRT_E_CUDA,
 * MCRT_E_OOM (messages on items[0].ctx). */
int mcrt_batch_create(const mcrt_batch_item *items, int n, const mcrt_solve_params *p,
                      const double *weights, int streams, mcrt_batch **out);
/* Replays the graph on cuda_stream with rays ray_offset .. ray_offset + N - 1 of
 * every cell (asynchronous).  The batch owns its scratch; the items' contexts
 * may be used for other solves between runs.  mcrt_set_fields on an item's
 * context (same grid) between runs is picked up by the next run; its proposal is
 * the one current in the context (valid and unbiased for any field).
 * mcrt_set_kdist on an item's context invalidates the batch. */
int mcrt_batch_run(mcrt_batch *b, uint64_t ray_offset, void *cuda_stream);
/* Waits for the last run; sums the items' counters; kernel_ms is the graph's
 * device time. */
int mcrt_batch_get_stats(mcrt_batch *b, mcrt_solve_stats *out);
const char *mcrt_batch_last_error(const mcrt_batch *b);
int mcrt_batch_destroy(mcrt_batch *b);

/* ---- learned proposal (no counterpart in the paper) ------------------------
 * The paper draws (n, g) from Zhang's T_max pdf (Section 2.1, Eqs. 13 and 16)
 * and directions isotropically (Eq. 9).  A learned proposal replaces both, per
 * emitting cell, by
 *   q(n,g) = (1 - mix) softmax(z)_(n,g) + mix p0(n,g),
 *   q(h)   = (1 - mix) softmax(z_up, z_down)_h + mix / 2   (h: sign of d_y),
 * where p0 is the plain pdf and z = MLP(features): 12 -> 64 -> 64 -> K + 2
 * with GELU activations, FP16 weights and FP32 arithmetic, K = n_bands n_g.
 * q is quantised to the integer counts of mcrt_set_cell_proposal and the ray
 * weight divides by the quantised probabilities, so Eq. 14 stays unbiased for
 * any weights; mix > 0 keeps every (n, g) that the plain pdf can draw drawable.
 * The network is trained on the GPU from tallies of plain solves to minimise
 * (E_q[Y^2] x E_q[steps per ray]) relative to the plain pdf, per cell:
 *   L = A(q) C(q) / (A(p0) C(p0)),  A(q) = sum_(k,h) m[k][h] / (q_k q_h),
 *   C(q) = c0 + sum_(k,h) c[k][h] q_k q_h,
 * with m and c the tallies of mcrt_tally_moments and c0 the fixed cost of a
 * ray in steps (cost == NULL: C = 1). */
enum { MCRT_NFEAT = 12, MCRT_NHIDDEN = 64 };
typedef struct mcrt_mlp mcrt_mlp;

/* Parameters of a network with K spectral outputs: theta = [W1 (64 x 12,
 * row-major output x input), b1 (64), W2 (64 x 64), b2 (64), W3 ((K+2) x 64),
 * b3 (K+2)]; output K is the upward hemisphere, K + 1 the downward one. */
int64_t mcrt_mlp_nparams(int K);
/* Creates a network for K = 1 .. 350 spectral points on `device` with all
 * parameters zero.  Errors: MCRT_E_ARG, MCRT_E_UNSUPPORTED (K > 350),
 * MCRT_E_CUDA, MCRT_E_OOM. */
int mcrt_mlp_create(int device, int K, mcrt_mlp **out);
/* Sets the FP32 master parameters (host [nparams]; the network runs with their
 * FP16 roundings) and the feature normalisation x = (f - mean) * inv_std (host
 * [12] each), and resets the Adam state.  Synchronous. */
int mcrt_mlp_set_params(mcrt_mlp *m, const float *theta, const float *feat_mean,
                        const float *feat_inv_std);
/* Copies the FP32 master parameters and, if theta_used != NULL, the FP16
 * values the network runs with (as floats) to host arrays [nparams].
 * Synchronous. */
int mcrt_mlp_get_params(mcrt_mlp *m, float *theta, float *theta_used);
/* Forward pass: feat (device [n][12]) -> q_out (device [n][K+2]): the mixed
 * spectral probabilities, then q_up and q_down.  p0: device plain
 * probabilities, [K] shared (p0_stride 0) or [n][K] (p0_stride K).
 * Asynchronous on cuda_stream. */
int mcrt_mlp_forward(mcrt_mlp *m, const float *feat, int64_t n, const float *p0, int p0_stride,
                     float mix, float *q_out, void *cuda_stream);
/* Loss modes: MCRT_LOSS_CELL, the mean over the batch of the per-cell ratio
 * A_c(q) C_c(q) / (A_c(p0) C_c(p0)); MCRT_LOSS_BATCH, the batch estimate of the
 * ratio of GPU time to a given relative error,
 *   (sum_c w_c A_c(q) / sum_c w_c A_c(p0)) (sum_c C_c(q) / sum_c C_c(p0)),
 * with sample weights w_c (1 / error scale^2 of the cell). */
enum { MCRT_LOSS_CELL = 0, MCRT_LOSS_BATCH = 1 };
/* Loss over a batch and its gradient.  Samples idx[0..n-1] (device, NULL:
 * 0..n-1) of a dataset of n_data samples: feat (device [n_data][12]), mom and
 * cost (device [n_data][K][2]; cost nullable: C = 1), p0 ([n_data][K],
 * p0_stride K, or [K], stride 0) and wgt (device [n_data], nullable: 1; used by
 * MCRT_LOSS_BATCH).  The gradient (FP32, [nparams]) goes to grad_out (device,
 * nullable) and to the network's own buffer; the loss is read by
 * mcrt_mlp_last_loss, which also reports (MCRT_E_ARG) an index outside
 * [0, n_data) -- such a sample is skipped, never read.  The gradient is reduced
 * in a fixed order: identical inputs give identical bits.  Asynchronous. */
int mcrt_mlp_loss_grad(mcrt_mlp *m, const float *feat, const float *mom, const float *cost,
                       float c0, const float *p0, int p0_stride, const float *wgt, int mode,
                       int64_t n_data, const int32_t *idx, int64_t n, float mix,
                       float *grad_out, void *cuda_stream);
/* One Adam step (Kingma & Ba 2015) of the master parameters with gradient grad
 * (device [nparams]; NULL: the network's last gradient); refreshes the FP16
 * copy.  Asynchronous. */
int mcrt_mlp_adam_step(mcrt_mlp *m, const float *grad, float lr, float beta1, float beta2,
                       float eps, void *cuda_stream);
/* Waits for the last mcrt_mlp_loss_grad and returns its loss. */
int mcrt_mlp_last_loss(mcrt_mlp *m, double *loss);
const char *mcrt_mlp_last_error(const mcrt_mlp *m);
int mcrt_mlp_destroy(mcrt_mlp *m);

/* The 12 features of cells (device int32 [n], linear index x fastest; NULL:
 * cells 0..n-1) into out (device float [n][12]): T_i/1000, x_i, y_c/h - 1
 * (h = ly/2), T_wall/1000 (two), eps of the nearer wall, h dT/dy / 1000
 * (centred, one-sided at the walls), h |grad_xz T| / 1000 (centred, periodic),
 * mean and standard deviation of T over the 3x3x3 neighbourhood (periodic in
 * x, z, cut at the walls) / T_i, the Planck-mean absorption coefficient at
 * (T_i, x_i) times h, T_max / T_i (T_max of Eq. 13).  Synchronous.  Errors:
 * MCRT_E_ARG (an index outside the grid; its row is NaN), MCRT_E_STATE,
 * MCRT_E_UNSUPPORTED (more than 512 T nodes). */
int mcrt_cell_features(mcrt_ctx *ctx, const int32_t *cells, int64_t n, float *out,
                       void *cuda_stream);
/* An FP32 solve of the whole grid (p->use_box must be 0) that also tallies,
 * for the listed cells (device int32 [n]), per spectral point k = n n_g + g and
 * hemisphere h (0: d_y > 0):
 *   mom_out [n][K][2]:  (1/N) sum of Y^2 p_k p_h over the rays that drew (k, h),
 *   cost_out [n][K][2]: (1/N) sum of steps / (p_k p_h) over the same rays,
 * with p the probabilities the rays were drawn with (plain or cell proposal).
 * sum m / (q_k q_h) and sum c q_k q_h are unbiased estimates of the second
 * moment of Y and of the medium steps per ray under any other proposal q.
 * q_out / sigma_out (device, nullable) receive the solve's Q and sigma.
 * Synchronous.  Errors as mcrt_solve_qrad, MCRT_E_UNSUPPORTED for K > 1024. */
int mcrt_tally_moments(mcrt_ctx *ctx, const mcrt_solve_params *p, const int32_t *cells, int64_t n,
                       float *mom_out, float *cost_out, double *q_out, double *sigma_out,
                       void *cuda_stream);
/* The plain pdf p0(n, g) of the current fields (Eq. 16 at T_max, as quantised)
 * to a host array [K].  Synchronous. */
int mcrt_get_plain_probs(mcrt_ctx *ctx, float *p0);
/* Quantises per-cell probabilities q (device [ncells][K+2]: spectral points,
 * then q_up; the last entry is ignored) into the cell proposal used by
 * MCRT_PROPOSAL_CELL solves: band counts from the sums over g, g counts within
 * each band, each a count of 2^32 proportional to its weight with at least one
 * count for every positive weight and the remainder on the first largest
 * weight; hemisphere count round(q_up 2^23) in [1, 2^23 - 1].  Synchronous.
 * Errors: MCRT_E_ARG (a row without positive weight), MCRT_E_STATE. */
int mcrt_set_cell_proposal_probs(mcrt_ctx *ctx, const float *q, void *cuda_stream);
/* Spectral proposals at each cell's own temperature (the classic ERMC draw,
 * Section 2: the paper replaces it by Zhang's T_max proposal, Eq. 13, because
 * its variance is large in cold cells).  MCRT_SPECTRAL_LOCAL: p_c(n,g) ~
 * w_g B_n(T_i) kappa_(n,g)(T_i), the emission spectrum of cell i.
 * MCRT_SPECTRAL_HYBRID: (1 - lam) p0 + lam p_local with p0 the T_max proposal
 * and lam = (T_i - T_min) / (T_max - T_min) clamped to [0, 1] (the cold cells
 * draw like the paper, the hottest ones like the classic ERMC).  Hemispheres
 * 1/2 each.  Quantised like mcrt_set_cell_proposal_probs (so every estimate
 * stays unbiased); later solves use it with MCRT_PROPOSAL_CELL.  Synchronous.
 * Errors: MCRT_E_ARG (bad mode), MCRT_E_STATE. */
enum { MCRT_SPECTRAL_LOCAL = 0, MCRT_SPECTRAL_HYBRID = 1 };
int mcrt_set_spectral_proposal(mcrt_ctx *ctx, int mode, void *cuda_stream);
/* Copies the current cell proposal to host arrays cn [ncells][nb],
 * cg [ncells][nb][ng], hemi [ncells].  Synchronous. */
int mcrt_get_cell_proposal(mcrt_ctx *ctx, uint64_t *cn, uint64_t *cg, uint32_t *hemi);
/* Features of every cell -> network -> mixture with the plain pdf (0 < mix <= 1)
 * -> cell proposal, all on the device; later solves use it with
 * MCRT_PROPOSAL_CELL.  The result equals mcrt_set_cell_proposal_probs of
 * mcrt_mlp_forward of mcrt_cell_features.  Synchronous.  Errors: MCRT_E_ARG
 * (K of the network differs from n_bands n_g, mix outside (0, 1]),
 * MCRT_E_STATE. */
int mcrt_set_learned_proposal(mcrt_ctx *ctx, mcrt_mlp *m, float mix, void *cuda_stream);

/* Machine ceilings the traversal is measured against (not part of the method).
 * A march step evaluates one exponential (the segment transmissivity, Eq. 10)
 * and gathers the {T, x} of the cell it enters plus two table entries; these
 * probes measure the GPU's rates for exactly those two operations.  Each call
 * allocates its own device memory on `device`, times one probe kernel with CUDA
 * events after one untimed launch, frees the memory and returns (synchronous;
 * no context needed).
 *
 * mcrt_probe_ex2: base-2 exponentials of the special-function unit
 * (ex2.approx.ftz.f32) per second over the whole GPU, every thread of a
 * full-occupancy grid running 8 independent chains x <- 2^(-x).  *sm_mhz is
 * the mean SM clock during the probe (SM cycles over global-timer time).
 *
 * mcrt_probe_gather: random 8-byte loads per second from a buffer of `bytes`
 * bytes (a power of two, 2^12 .. 2^35), 8 independent loads in flight per
 * thread of a full-occupancy grid, indices from per-load 32-bit congruential
 * generators, so the lanes of a warp hit different sectors: the worst case of
 * the march's gathers.  Useful bytes per second = 8 * *per_s.
 *
 * Errors: MCRT_E_ARG (NULL output, bytes out of range or not a power of two),
 * MCRT_E_OOM, MCRT_E_CUDA (no such device, launch failure). */
int mcrt_probe_ex2(int device, double *per_s, double *sm_mhz);
int mcrt_probe_gather(int device, uint64_t bytes, double *per_s);

/* Releases all device memory of the context; NULL is accepted.  Waits for the
 * context's outstanding work. */
int mcrt_destroy(mcrt_ctx *ctx);

/* Static description of a status code. */
const char *mcrt_status_string(int status);

/* Message of the last error raised on this context (empty if none). */
const char *mcrt_last_error(const mcrt_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* MCRT_H */
