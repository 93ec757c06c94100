/*
 * mcrt_oracle.h -- TEST INFRASTRUCTURE ONLY (not part of the product).
 *
 * Plain FP64 CPU oracle of the emission-based reciprocal Monte Carlo (ERMC)
 * estimator of the radiative source Q_rad (Silvestri & Pecnik, arXiv:1810.00188,
 * Section 2, Eqs. 1-17, Algorithm 1).  Only the tests, the package smoke check and
 * the CPU-baseline leg of the benchmark load it.  It shares no code with the CUDA
 * library.
 */
#ifndef MCRT_ORACLE_H
#define MCRT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int nx, ny, nz;            /* cells; y wall-normal, x and z periodic            */
  double lx, ly, lz;         /* box lengths [m]                                   */
  const double *T;           /* [nz][ny][nx] temperature [K]                      */
  const double *xh2o;        /* [nz][ny][nx] H2O mole fraction, NULL = x_ref      */
  double eps_wall[2];        /* emissivity of the y=0 and y=ly walls              */
  double T_wall[2];          /* temperature of the walls [K]                      */
  int reflect;               /* 0 diffuse, 1 specular                             */
  int n_bands, n_g;
  const double *w_g;         /* [n_g] quadrature weights                          */
  double T0, dT;
  int nT;
  const double *kappa;       /* [n_bands][n_g][nT] at x_ref [1/m]                 */
  const double *B;           /* [n_bands][nT] band blackbody intensity            */
  double x_ref;
  /* Wall-normal face coordinates y_0 = 0 < y_1 < ... < y_ny = ly of a stretched
   * grid (the channel DNS grids of Section 5), or NULL for uniform cells.  x and
   * z stay uniform. */
  const double *yf;
  /* 0: x and z periodic (the channel); 1: black walls on the x = 0, x = lx,
   * z = 0 and z = lz faces too, at temperatures T_xz[0..3] (the closed 3D
   * boxes of the paper's verification cases 3 and 4, Table 1) */
  int xz_walls;
  double T_xz[4];
} orc_problem;

typedef struct {
  int rays_per_cell;
  uint64_t ray_offset;
  uint64_t seed;
  uint32_t snapshot;
  double tol;                /* transmissivity cut-off                            */
  int max_steps;             /* cap on medium segments per ray                    */
  int origin;                /* 0 uniform in the cell, 1 cell centre              */
  int use_box;               /* 0: whole grid; 1: box below (half-open ranges)    */
  int box[6];                /* i0,i1,j0,j1,k0,k1                                 */
  int nthreads;              /* <= 0: one                                         */
  /* Optional per-cell proposal (NULL: the global Planck-T_max proposal).        */
  const uint64_t *cell_cn;   /* [ncells_box][n_bands] cumulative counts of 2^32   */
  const uint64_t *cell_cg;   /* [ncells_box][n_bands][n_g]                        */
  const uint32_t *cell_hemi; /* [ncells_box] upward-hemisphere count of 2^23      */
  /* Optional second-moment tallies per emitting cell, spectral point and
   * hemisphere (NULL: none): tally[b][(n n_g + g) 2 + h] = (1/N) sum over the
   * rays r of cell b that drew (n, g, h) of Y_r^2 p(n,g) p(h), where p are the
   * probabilities the ray was drawn with and h = 0 is the upward (d_y > 0)
   * hemisphere.  Summed over h and (n,g) with weights 1/(q(n,g) q(h)) it is the
   * unbiased estimate of E[Y^2] under another proposal q. */
  double *tally;
  /* Optional cost tallies, same layout: (1/N) sum over those rays of
   * steps_r / (p(n,g) p(h)); weighted by q(n,g) q(h) and summed it is the
   * unbiased estimate of the mean medium segments per ray under q. */
  double *tally_cost;
  /* Multigrid (Section 4.3): number of overlaid grids (0 or 1: the problem's
   * grid only) and the segments a ray marches on each grid before it falls onto
   * the next coarser one.  Grid l + 1 halves every dimension of grid l and holds
   * the mean T and x of its 2x2x2 children; it exists while every dimension of
   * grid l is even and halves to at least 3 (orc_mg_max_levels). */
  int mg_levels;
  int mg_steps;
} orc_params;

typedef struct {             /* per emitting cell of the box, x fastest           */
  double *sum_y;             /* sum_r Y_r                                         */
  double *sum_y2;            /* sum_r Y_r^2                                       */
  double *sum_abs;           /* sum_r w_r sum|terms_r|   (parity scale)           */
  double *sum_wall;          /* sum_r w_r (wall terms of ray r)                   */
  double *sum_wall2;         /* sum_r (w_r wall_r)^2                              */
  uint64_t *steps;           /* medium segments                                   */
  uint64_t *capped;          /* rays stopped by max_steps                         */
} orc_cell_sums;

typedef struct {
  int n, g;                  /* band and quadrature point                         */
  int cell[3];               /* start cell i,j,k                                  */
  double frac[3];            /* start position inside the cell, in [0,1]          */
  double dir[3];             /* unit direction                                    */
  double tol;
  int max_steps;
  uint64_t seed;             /* Philox identity for reflection draws              */
  uint32_t ray;
  uint32_t snapshot;
} orc_ray_in;

typedef struct {
  double X;                  /* sum of kappa_i (B_i - B_j) tau alpha + walls + residual */
  double abs_terms;
  double X_wall;
  double tau_end;
  int64_t steps;
  int capped;
  int walls;                 /* wall events                                       */
  double path;               /* geometric path length travelled                   */
} orc_ray_out;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_uniform(uint32_t w);
double orc_interp(const double *v, double T0, double dT, int nT, double T);
int orc_quantize(const double *w, int K, uint64_t *cum);
int orc_plain_proposal(const orc_problem *P, uint64_t *cn, uint64_t *cg, double *T_max);
int orc_trace_ray(const orc_problem *P, const orc_ray_in *in, orc_ray_out *out);
int orc_mg_max_levels(int nx, int ny, int nz);
/* One ray as orc_trace_ray, marched on mg_levels overlaid grids with mg_steps
 * segments per grid (Section 4.3). */
int orc_trace_ray_mg(const orc_problem *P, const orc_ray_in *in, int mg_levels, int mg_steps,
                     orc_ray_out *out);
int orc_solve(const orc_problem *P, const orc_params *S, orc_cell_sums *out);
/* Absorption-based reciprocal estimate over the whole grid (every cell emits):
 * per batch k = r mod K and cell, the deposits of the rays of batch k into the
 * cell (acc [K][nc], zeroed by the caller), their absolute sum (absacc [nc]),
 * optionally the emission-based sums of each cell's own samples per batch
 * (accE [K][nc] or NULL) and each cell's own medium segments (steps [nc]).
 * Single grid only. */
int orc_solve_armc(const orc_problem *P, const orc_params *S, int K, double *acc, double *absacc,
                   double *accE, uint64_t *steps);
int orc_exchange(const orc_problem *P, const orc_params *S, double *G, double *G2,
                 double *Gw, double *Gw2);
/* ---- learned proposal (no counterpart in the paper; replaces the pdf of
 * Eqs. 13, 16 per emitting cell) -- see learn_oracle.c ---------------------- */
enum { ORC_NFEAT = 12, ORC_HIDDEN = 64 };
int orc_features(const orc_problem *P, const int32_t *cells, int64_t n, double T_max,
                 double *out);
int64_t orc_mlp_nparams(int K);
int orc_mlp_forward(const double *theta, int K, const double *fmean, const double *finv,
                    const double *feat, int64_t n, const double *p0, int p0_stride,
                    double mix, double *q);
int orc_mlp_loss_grad(const double *theta, int K, const double *fmean, const double *finv,
                      const double *feat, const double *m, const double *cst, double c0,
                      const double *p0, const double *wgt, int mode, int64_t n, double mix,
                      double *loss, double *grad);
void orc_adam(double *theta, const double *grad, double *m1, double *m2, int64_t n, double lr,
              double beta1, double beta2, double eps, int t);
int orc_learned_counts(const double *q, int nb, int ng, double q_up, uint64_t *cn,
                       uint64_t *cg, uint32_t *hemi);
int orc_spectral_proposal(const orc_problem *P, int mode, double T_min, double T_max,
                          const double *p0, const int32_t *cells, int64_t n, double *q_out);

int orc_quadrature(const orc_problem *P, const double *mu, const double *mu_w, int nmu,
                   int nphi, const double *vn, const double *vw, int nv, int origin,
                   double tol, int max_steps, const int *cells, int ncq, int nthreads,
                   double *q);

#ifdef __cplusplus
}
#endif
#endif
