// Internal interface between the C-ABI host code (mcrt_api.cpp) and the CUDA
// kernels (trace.cu, fields.cu).  Not installed; not part of the ABI.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace mcrt {

// State of a long ray handed from the FP32 trace kernel to the warp-parallel
// march (long_rays.cu), taken between two segments: the parametric axes
// (crossing m of an axis at fma(m, ts, t0)), the next crossings, the current
// cell, the running transmissivity and sum, and the ray's identity (sample slot,
// Philox words, snapshot of a batch).  128 bytes, written and read as float4s.
struct __align__(16) LongRay {
  float t0x, t0y, t0z, tsx;
  float tsy, tsz, cntx, cnty;
  float cntz, tnx, tny, tnz;
  float tprev, tau, X, B_i;
  float B_last, scale;
  unsigned krow, n;          // table row of (n, g) and the band
  int ix, iy, iz;
  unsigned signs;            // (sx + 1) | (sy + 1) << 2 | (sz + 1) << 4
  unsigned lin, slot, r, ray;  // cell, sample slot, ray index in the cell, Philox ray word
  unsigned cellid, steps, nrefl, snap;  // emitting cell, segments so far, reflections, batch snapshot
};
static_assert(sizeof(LongRay) == 128, "LongRay is eight float4");

// Entries of a solve's device counters (see TraceArgs::counters).
constexpr int NCOUNTERS = 10;

// Everything one trace launch reads.  Device pointers only.
// One snapshot of a batched FP32 solve (one persistent launch over many
// fields that share the k-distribution): what differs from snapshot to
// snapshot.  Snapshot k owns the global brick-order positions [p0, next p0).
struct SnapArgs {
  const uint2 *fpos32;               // positions of every multigrid grid
  const float *yf32;                 // stretched faces or null
  const float *bwall32;              // [2][nb]
  const float *wgt32;                // plain-proposal ray weights [nb*ng]
  const unsigned long long *cn, *cg; // plain proposal counts
  const unsigned short *guide;
  const unsigned long long *cell_cn, *cell_cg;  // per-cell proposal or null
  const unsigned int *cell_hemi;
  double *q, *sigma;                 // outputs, the whole grid
  long long p0;                      // first global position
  int nx, ny, nz, reflect;
  float dx, dy, dz, eps0, eps1;
  unsigned snapshot;                 // fourth Philox counter word
};

struct TraceArgs {
  // grid (uniform cells; y wall-normal; x, z periodic)
  int nx, ny, nz;
  double dx, dy, dz;
  // tables on uniform T nodes: T0 + t/inv_dT
  int nb, ng, nT;
  double T0, inv_dT, inv_xref;
  double eps_wall[2];
  int reflect;  // 0 diffuse, 1 specular
  // stretched wall-normal grid: the ny + 1 faces (null: uniform dy)
  const double *yf64;
  const float *yf32;
  // closed box: black walls on the x and z faces (bwall rows 2..5: x = 0,
  // x = lx, z = 0, z = lz) instead of periodic x and z
  int xz_walls;
  // batched launch: some snapshot has stretched y faces (the kernel's general variant)
  int batch_stretched;
  // device data; the *32 / *64 members are used by the FP32 / FP64 kernel
  const uint2 *fpos32;      // FP32 kernel: {(node << 23) | fraction * 2^23, bits of x / x_ref}
  const double2 *field64;
  const float2 *ktab32;     // [nb*ng][nT] {kappa_t, kappa_{t+1} - kappa_t} at x_ref
  const double2 *ktab64;
  const float2 *btab32;     // [nb][nT] {B_t, B_{t+1} - B_t}
  const float4 *kbtab32;    // [nb*ng][nT] {kappa_t, its slope, B_t of band n, its slope}:
                            // one 16-byte load per march step
  const double2 *btab64;
  const float *bwall32;     // [6][nb] wall band intensity: y = 0, y = ly, x = 0, x = lx, z = 0, z = lz
  const double *bwall64;
  const double *w_g;        // [ng]
  const float *wgt32;       // [nb*ng] plain-proposal ray weight w_g / (p q), host FP64 -> FP32
  const float *w_g32;       // [ng] quadrature weights in FP32
  const unsigned long long *cn;       // [nb] cumulative counts of 2^32 (plain proposal)
  const unsigned long long *cg;       // [nb*ng]
  const unsigned long long *cell_cn;  // per-cell proposal [ncells][nb] or null
  const unsigned long long *cell_cg;  // [ncells][nb*ng]
  const unsigned int *cell_hemi;      // [ncells] count of 2^23, or null (plain: 2^22)
  int counts_in_smem;                 // bit 0: plain counts staged in shared memory (<= 48 KB);
                                      // bit 1: per-cell counts staged per warp (<= 48 KB)
  const unsigned short *guide;        // [fp32_guide_size()] guide table of the plain band counts
  const unsigned char *gguide;        // [nb][fp32_gguide_size()] the plain g counts' guides
  // FP32 kernel: brick-order positions [chunk_p0, chunk_p1) of this launch, the
  // per-ray sample scratch [(p - chunk_p0) * rays + r] and per-position step sums
  long long chunk_p0, chunk_p1;
  float *ybuf;
  unsigned long long *step_acc;
  // per-ray step counts, same indexing as ybuf (null: not stored); read by the
  // second-moment tally of the learned proposal
  unsigned *ray_steps;
  // batched runs: ray_offset read from device memory (set before each graph
  // replay) when non-null; persistent grid size override (0: one full wave)
  const unsigned long long *ray_offset_dev;
  int grid_blocks;
  // batched FP32 solve: the snapshots (device [nsnaps + 1]; the last entry only
  // holds the end position in p0); null for a single solve
  const SnapArgs *snaps;
  int nsnaps;
  // multigrid (Section 4.3): grids used (1: exact march) and segments per grid;
  // the fields of grid l (l >= 1) follow those of grid l - 1 in field64 / fpos32
  int mg_levels, mg_steps;
  // FP32 exact march: hand-off of long rays to the warp-parallel march (count in
  // counters[7]); long_rays null or long_steps 0: never
  LongRay *long_rays;
  int long_cap;      // entries of long_rays
  int long_steps;    // segments marched before a hand-off
  float long_flight; // x/z crossings left in the flight for a hand-off
  int claim_rays;    // FP32 kernels: rays per claimed run of cells (<= 0: 1024)
  // solve
  int rays, max_steps, origin;
  double tol;
  // the FP32 kernels' copies of tol, the cell sizes and the wall emissivities,
  // rounded once on the host: the kernels read them where they are used instead
  // of converting the binary64 members there (a conversion on the narrow binary64
  // pipe each time the compiler rematerialises the value)
  float tol32, dx32, dy32, dz32, eps32[2];
  unsigned int key0, key1, snapshot;
  // the Philox round keys of (key0, key1), for philox10r (set_round_keys)
  unsigned int rkey[20];
  unsigned long long ray_offset;
  int bi0, bj0, bk0, bnx, bny, bnz;
  long long ncells_box;
  // outputs (box-sized)
  double *q, *sigma;
  unsigned long long *steps_cell;
  // FP32 kernels: per-cell tallies in binary32 pairs (1) instead of binary64 (0);
  // binary64 tallies read by plain loads (1) instead of the TMA-fed kernel (0)
  int tally32, reduce_plain;
  // binary64 tallies of more than one segment (tally_segments): each segment's
  // sums by a warp of their own, [segment][chunk position] {sum y, sum y^2},
  // then added in order by a second kernel (null: one warp adds a cell's
  // segments in order; the same bits)
  double2 *tally_part;
  // absorption-based estimate (null: off): per-batch binary64 sums [16][armc_nc]
  // of the deposits into each cell and of each cell's own samples
  double *armc_acc, *ermc_acc;
  long long armc_nc;
  unsigned long long *counters;  // [0] steps [1] capped [2] wall hits [3] rays [4] longest ray (steps)
                                 // [5] error flags [6] FP32 kernel: claimed positions
                                 // [7] long rays handed off by this launch
                                 // [8] long rays finished by the warp-parallel march
                                 // [9] long rays that found the buffer full (NCOUNTERS entries)
};

// Segments of the binary64 per-cell tally (Eq. 8).  A cell's N samples form
// tiles of 32; its sums are the compensated sum, in order, of the sums of
// consecutive runs of tally_seg_len tiles, each itself a compensated sum of the
// runs' exact tile sums in order.  The split depends on N alone (up to
// TALLY_SEG_TILES tiles per run, runs of equal length but for the last), so any
// kernel that follows it gives the same bits; N <= 32 TALLY_SEG_TILES is one run.
constexpr int TALLY_SEG_TILES = 64;
__host__ __device__ inline int tally_segments(int ntile) {
  return ntile > 0 ? (ntile + TALLY_SEG_TILES - 1) / TALLY_SEG_TILES : 0;
}
__host__ __device__ inline int tally_seg_len(int ntile) {
  const int n = tally_segments(ntile);
  return n > 0 ? (ntile + n - 1) / n : 0;
}

// Largest grid of the grid-stride kernels (reductions, packing, coarsening): 16
// CTAs per SM of the current device (its SM count read once per device).
long long grid_stride_blocks();

// Multigrid grid count of an nx x ny x nz grid and the cells of all its grids.
int multigrid_levels(int nx, int ny, int nz);
long long multigrid_cells(int nx, int ny, int nz, int levels);
// Fields of grid l + 1 (2x2x2 means of T and x) from grid l of n0 x n1 x n2 cells.
// On a stretched grid (yf non-null) the means are weighted by the children's
// heights; `level` is grid l, whose face F is yf[F << l].
cudaError_t launch_coarsen(const double2 *fine, int n0, int n1, int n2, double2 *coarse,
                           const double *yf, int level, cudaStream_t s);

// Simple kernel: one warp per cell, lane-strided rays (FP64 parity mode).
cudaError_t launch_trace(const TraceArgs &a, int precision, cudaStream_t s);
// FP32 kernel with converged initialisation and lane refill, the warp-parallel
// march of the long rays it handed off (when long_rays_on), then the per-cell
// reduction (trace_fp32.cu); two or three launches per chunk.  min_blocks:
// occupancy target (1-4 CTAs of 256 threads per SM); steps_per_round: march
// steps between refills of idle lanes (1, 2, 4).
// marks (nullable): four events recorded on s before the trace kernel, after it,
// after the long-ray march (right after the trace kernel when there is none) and
// after the reduction.
// kernels (nullable): the number of kernels launched.
cudaError_t launch_trace_fp32(const TraceArgs &a, int min_blocks, int steps_per_round,
                              cudaStream_t s, cudaEvent_t *marks = nullptr, int *kernels = nullptr);
// The binary64 per-cell tallies of one FP32 solve chunk with the samples
// streamed by TMA (tally_tma.cu; the same results as reduce_cells_kernel).
// Launches nothing and leaves *launched false when the samples' layout does not
// allow the tiled copy (rays % 4 != 0) or the driver has no tensor-map encoder.
// *kernels: the kernels it launched (0: none, the caller then tallies by plain
// loads; 2 when the segments of each cell are summed by warps of their own,
// a.tally_part non-null, and added by a second kernel).
cudaError_t launch_reduce_tma(const TraceArgs &a, cudaStream_t s, int *kernels);
// The second kernel of a split binary64 tally (either reader): adds each cell's
// segment sums in a.tally_part in order and writes Q, sigma and the step counts.
cudaError_t launch_combine_segments(const TraceArgs &a, cudaStream_t s);
// Q and sigma of the absorption-based estimate (hybrid = 0) or of its
// temperature-weighted combination with the emission-based one (hybrid = 1) from
// the per-batch sums of the AR trace launches; K batches of N rays per cell.
cudaError_t launch_armc_finalize(const double *acc, const double *eacc, long long nc, int K, int N,
                                 int hybrid, const double2 *field, double T_min, double T_max, double *q,
                                 double *sigma, cudaStream_t s);
long long fp32_bricks_positions(int bnx, int bny, int bnz);
// The warp-parallel march of the long rays the last FP32 trace launch handed off
// (a.long_rays[0 .. min(counters[7], long_cap))); writes their samples and adds
// their counts.  Launched after each trace launch, before the reduction.
cudaError_t launch_long_rays(const TraceArgs &a, cudaStream_t s);
// Entries of the long-ray buffer for a launch of `rays` rays and the hand-off
// threshold long_steps.
long long long_ray_capacity(long long rays, int long_steps);
// True when a launch with these arguments hands long rays off (exact march,
// periodic x and z, a buffer and a threshold).
inline bool long_rays_on(const TraceArgs &a) {
  return a.long_rays && a.long_cap > 0 && a.long_steps > 0 && a.long_steps < 0x7fffffff &&
         a.mg_levels <= 1 && !a.xz_walls;
}
// Batched FP32 solve over a.snaps: trace + reduce of the global positions
// [chunk_p0, chunk_p1), one persistent launch each.
cudaError_t launch_trace_fp32_batch(const TraceArgs &a, int min_blocks, int steps_per_round,
                                    cudaStream_t s);
cudaError_t prepare_trace_fp32_batch(int min_blocks, int steps_per_round, int nb, int ng, int nsnaps,
                                     int counts_in_smem, int multigrid, int *blocks_per_sm, int *num_sms);
int fp32_batch_max_snapshots();
// Sets the launch attributes of the chosen FP32 variant and returns its
// resident CTAs per SM (call before stream capture).
cudaError_t prepare_trace_fp32(int min_blocks, int steps_per_round, int nb, int ng, int counts_in_smem,
                               int multigrid, int *blocks_per_sm, int *num_sms);
int fp32_brick_volume();
int fp32_cell_stage_fits(int nb, int ng);
int fp32_guide_size();
int fp32_guide_bits();  // guide[m] covers R_n in [m, m + 1) 2^(32 - bits)
int fp32_gguide_size();  // g guide entries per band
int fp32_gguide_bits();
// the plain proposal's counts, guide and g guides fit the FP32 kernel's shared staging
int fp32_plain_stage_fits(int nb, int ng);

// Static device scratch of the allocation-free solve (noalloc.cu): its size,
// and its device address on `device` (the current device), looked up once per
// device.
size_t noalloc_scratch_bytes();
cudaError_t noalloc_scratch(int device, void **out);

// Packs T (and x, or x_ref where x is null) into the FP64 and FP32 field
// layouts and reduces {max T, min T, bad count}.  stats: [0] max T bits (u64),
// [1] min T bits (u64), [2] count of rejected cells.
// Packs each cell's interpolation position for the FP32 kernel (nT <= 512).
cudaError_t launch_pack_positions(const double2 *f64, long long n, double T0, double inv_dT, int nT,
                                  double inv_xref, uint2 *pos, cudaStream_t s);

// ---- learned proposal (learn.cu) ----
constexpr int kNFeat = 12, kNHidden = 64;
constexpr int kMaxTrainOut = 352;   // n_out (spectral points + 2) limit of the training kernel
constexpr int kMaxTallyK = 1024;    // spectral points limit of the tally kernel

struct FeatArgs {
  int nx, ny, nz;
  double dx, dy, dz, h;
  const double *yf;  // stretched grid: the ny + 1 wall-normal faces (null: uniform dy)
  double T_wall[2], eps_wall[2], T_max;
  const double2 *field64;
  const uint2 *fpos32;
  // Planck-mean absorption per T node as a rational function of the fraction fr
  // towards the next node: [2 t] = {N0, N1, N2, D0}, [2 t + 1] = {D1, 0, 0, 0},
  // kappa_P = (N0 + N1 fr + N2 fr^2) / (D0 + D1 fr) at x_ref
  const float4 *kptab;
  int nT;
  const int *cells;  // null: cells 0..n-1
  long long n;
  float *out;        // [n][12]
  unsigned long long *err;
};
cudaError_t launch_features(const FeatArgs &f, cudaStream_t s);

struct TallyArgs {
  const int *cells;
  long long n;
  int nx, ny, nz;
  long long chunk_p0, chunk_p1;
  const float *ybuf;
  const unsigned *ray_steps;
  int N;
  unsigned key0, key1, snapshot;
  unsigned long long ray_off;
  const unsigned long long *cn, *cg;            // plain proposal
  const unsigned long long *cell_cn, *cell_cg;  // or per-cell proposal
  const unsigned *cell_hemi;
  int nb, ng;
  float *m_out, *c_out;  // [n][nb*ng][2]
  unsigned long long *err;
};
cudaError_t launch_tally(const TallyArgs &t, cudaStream_t s);

// theta layout: W1 [64][12], b1 [64], W2 [64][64], b2 [64], W3 [K+2][64], b3 [K+2]
long long mlp_nparams(int K);

struct MlpInferArgs {
  const __half *theta16;
  const float *fmean, *finv;  // [12]
  int K;
  const float *feat;          // [n][12]
  long long n;
  const float *p0;            // [K] (p0_stride 0) or [n][K]
  int p0_stride;
  float mix;
  float *q_out;               // [n][K+2]: probabilities (spectral points, then the hemispheres)
  int nb, ng;
  unsigned long long *err;
};
cudaError_t launch_mlp_infer(const MlpInferArgs &a, cudaStream_t s);

// Quantises per-cell probabilities q [n][K+2] (spectral points, then q_up) into
// cumulative counts (same rule as the host's plain proposal).
// Per-cell spectral proposals at the cells' own temperatures (learn.cu):
// mode 0 the local emission spectrum, 1 the temperature-weighted mix with the
// T_max proposal p0.
struct SpectralArgs {
  long long n;
  int nb, ng, nT, mode;
  double T_min, T_max;
  const uint2 *fpos32;
  const double2 *field64;
  const float2 *ktab32, *btab32;
  const float *w_g32, *p0;
  unsigned long long *cell_cn, *cell_cg;
  unsigned *cell_hemi;
  unsigned long long *err;
};
cudaError_t launch_spectral_proposal(const SpectralArgs &a, cudaStream_t s);
cudaError_t launch_quantize_cells(const float *q, long long n, int nb, int ng,
                                  unsigned long long *cell_cn, unsigned long long *cell_cg,
                                  unsigned *cell_hemi, unsigned long long *err, cudaStream_t s);

struct MlpTrainArgs {
  const __half *theta16;
  const float *fmean, *finv;
  int K;
  const float *feat, *mom, *cost;  // [N][12], [N][K][2], [N][K][2] or null
  float c0;
  const float *p0;                 // [N][K] or [K]
  int p0_stride;
  const float *wgt;                // [N] sample weights (mode 1), or null (1)
  int mode;                        // 0: mean per-cell work ratio; 1: batch time ratio
  int pass;                        // mode 1: 0 = batch sums only, 1 = gradient
  const double *bsum;              // mode 1 pass 1: {sum w A(q), sum w A(p0), sum C(q), sum C(p0)}
  double *stat_partial;            // mode 1 pass 0: [grid][4]
  const int *idx;                  // batch -> sample, or null (sample = batch index)
  long long n_data;                // samples in the dataset (idx must stay below)
  long long n;                     // batch size
  float mix;
  float *partial;                  // [grid][nparams]
  double *loss_partial;            // [grid]
  int grid;
  unsigned long long *err;         // set when an index is outside the dataset
};
cudaError_t launch_mlp_train(const MlpTrainArgs &a, cudaStream_t s);
// Adds the CTAs' gradient partials in order; the loss is the sum of the loss
// partials, or (bsum non-null) the batch time ratio of the four batch sums.
cudaError_t launch_grad_reduce(const float *partial, const double *loss_partial, int grid,
                               long long np, const double *bsum, float *grad, double *loss,
                               cudaStream_t s);
cudaError_t launch_stat_reduce(const double *stat_partial, int grid, double *bsum, cudaStream_t s);
cudaError_t launch_adam(float *theta, __half *theta16, const float *grad, float *m1, float *m2,
                        long long np, float lr, float beta1, float beta2, float eps, float c1,
                        float c2, cudaStream_t s);
cudaError_t launch_theta_to_half(const float *theta, __half *theta16, long long np, cudaStream_t s);
int mlp_train_grid();

cudaError_t launch_pack_fields(const void *T, const void *x, int fp64_in, double x_ref,
                               long long n, double2 *f64,
                               unsigned long long *stats, cudaStream_t s);

}  // namespace mcrt
