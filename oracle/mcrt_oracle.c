/*
 * mcrt_oracle.c -- TEST INFRASTRUCTURE ONLY (not part of the product).
 *
 * Plain, slow, FP64 CPU oracle of the emission-based reciprocal Monte Carlo
 * (ERMC) estimator of the radiative source Q_rad [W/m^3] of Silvestri & Pecnik,
 * "A fast GPU Monte Carlo radiative heat transfer implementation for coupling
 * with direct numerical simulation" (arXiv:1810.00188).  It follows the paper's
 * Section 2 (Eqs. 1-17) and the CPU Algorithm 1 step by step and consumes the same
 * counter-based random draws as the CUDA library, so the two can be compared
 * draw for draw.  It shares no code with the library.  Only the tests, the
 * package smoke check and the CPU-baseline leg of the benchmark load it.
 *
 * Readings of the paper taken here (the paper is silent or ambiguous):
 *  - random numbers: Philox4x32-10 keyed by (cell, ray, draw block, snapshot),
 *    uniforms from the top 23 bits of a word, U = (w>>9 + 1/2) 2^-23 (exact in
 *    binary32 and binary64);
 *  - the polar axis of the direction (Eq. 9) is y, the wall normal;
 *  - the ray origin is uniform in the cell (f_V = 1/V_i, Eq. 4), or the cell
 *    centre (Algorithm 1) on request;
 *  - (n, g) are drawn with two words against integer cumulative counts of 2^32
 *    built from the discrete pdfs f_n and f_g(n) of Eq. 16 at T_max (Eq. 13), and
 *    the ray weight uses those exact quantised probabilities;
 *  - one axis is crossed per step (lowest axis on exact ties);
 *  - the residual dump after the cut-off uses the last medium cell's B;
 *  - grey walls absorb eps_w of the ray and reflect the rest diffusely (or
 *    specularly on request); Eq. 3 multiplies tau by (1 - eps_w) per reflection.
 *
 * Pins (tests/test_oracle_*.py): exponential-integral closed forms of grey and
 * non-grey isothermal slabs (black, grey-diffuse and grey-specular walls), the
 * optically thin limit, an independent segment-list path integral in 3D,
 * energy conservation, reciprocity, deterministic quadrature, statistical
 * tests of the generator and properties of the quantised pdfs.
 */
#include "mcrt_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdatomic.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) --------------------- */

static void philox_round(uint32_t c[4], const uint32_t k[2]) {
  const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
  const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
  const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
  const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
  const uint32_t n0 = hi1 ^ c[1] ^ k[0];
  const uint32_t n2 = hi0 ^ c[3] ^ k[1];
  c[0] = n0;
  c[1] = lo1;
  c[2] = n2;
  c[3] = lo0;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  uint32_t k[2] = {key[0], key[1]};
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k[0] += 0x9E3779B9u;
      k[1] += 0xBB67AE85u;
    }
    philox_round(c, k);
  }
  memcpy(out, c, sizeof(c));
}

void orc_philox_batch(const uint32_t *ctr, int64_t n, const uint32_t key[2], uint32_t *out) {
  for (int64_t i = 0; i < n; ++i) orc_philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}

double orc_uniform(uint32_t w) { return ((double)(w >> 9) + 0.5) * 0x1p-23; }

static void draw(uint64_t seed, uint32_t cell, uint32_t ray, uint32_t block, uint32_t snap,
                 uint32_t out[4]) {
  const uint32_t ctr[4] = {cell, ray, block, snap};
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  orc_philox4x32_10(ctr, key, out);
}

/* ---- property tables (Section 2.2: linear interpolation in T) -------------- */

double orc_interp(const double *v, double T0, double dT, int nT, double T) {
  const double f = (T - T0) / dT;
  double t = floor(f);
  double frac;
  if (t < 0.0) {
    t = 0.0;
    frac = 0.0;
  } else if (t >= (double)(nT - 1)) {
    t = (double)(nT - 2);
    frac = 1.0;
  } else {
    frac = f - t;
  }
  const int it = (int)t;
  return v[it] + frac * (v[it + 1] - v[it]);
}

static double kappa_at(const orc_problem *P, int n, int g, double T, double x) {
  const double k = orc_interp(P->kappa + ((size_t)n * P->n_g + g) * P->nT, P->T0, P->dT, P->nT, T);
  return k * (x / P->x_ref); /* kappa proportional to the H2O mole fraction */
}

static double B_at(const orc_problem *P, int n, double T) {
  return orc_interp(P->B + (size_t)n * P->nT, P->T0, P->dT, P->nT, T);
}

static double x_of(const orc_problem *P, size_t c) { return P->xh2o ? P->xh2o[c] : P->x_ref; }

/* ---- discrete pdfs as integer counts of 2^32 (Eqs. 15-17) ------------------ */

/* counts m_k ~ 2^32 w_k / sum(w), every positive weight at least one count, the
 * rounding remainder given to the first largest weight; returns the cumulative
 * counts (last one = 2^32).  Returns -1 when no weight is positive. */
int orc_quantize(const double *w, int K, uint64_t *cum) {
  double W = 0.0;
  for (int k = 0; k < K; ++k) W += w[k];
  if (!(W > 0.0)) return -1;
  int kmax = 0;
  for (int k = 1; k < K; ++k)
    if (w[k] > w[kmax]) kmax = k;
  int64_t m[4096];
  if (K > 4096) return -2;
  int64_t total = 0;
  for (int k = 0; k < K; ++k) {
    if (w[k] > 0.0) {
      int64_t mk = (int64_t)floor((w[k] / W) * 4294967296.0);
      m[k] = mk < 1 ? 1 : mk;
    } else {
      m[k] = 0;
    }
    total += m[k];
  }
  m[kmax] += (int64_t)4294967296LL - total;
  uint64_t acc = 0;
  for (int k = 0; k < K; ++k) {
    acc += (uint64_t)m[k];
    cum[k] = acc;
  }
  return 0;
}

/* Zhang's T_max proposal (Eq. 13) discretised as Eq. 16: band pdf
 * f_n ~ B_n(T_max) sum_g w_g k_{n,g}(T_max), g pdf f_g(n) ~ w_g k_{n,g}(T_max).
 * T_max is the largest medium temperature or wall temperature of an emitting
 * wall.  A band with no absorption gets uniform g counts (it is never drawn). */
int orc_plain_proposal(const orc_problem *P, uint64_t *cn, uint64_t *cg, double *T_max) {
  double Tm = 0.0;
  const size_t N = (size_t)P->nx * P->ny * P->nz;
  for (size_t c = 0; c < N; ++c)
    if (P->T[c] > Tm) Tm = P->T[c];
  for (int w = 0; w < 2; ++w)
    if (P->eps_wall[w] > 0.0 && P->T_wall[w] > Tm) Tm = P->T_wall[w];
  if (P->xz_walls)
    for (int f = 0; f < 4; ++f)
      if (P->T_xz[f] > Tm) Tm = P->T_xz[f];
  if (T_max) *T_max = Tm;
  const int nb = P->n_bands, ng = P->n_g;
  double *wn = (double *)malloc(sizeof(double) * nb);
  double *wg = (double *)malloc(sizeof(double) * ng);
  int rc = 0;
  for (int n = 0; n < nb && rc == 0; ++n) {
    double s = 0.0;
    for (int g = 0; g < ng; ++g) {
      wg[g] = P->w_g[g] * orc_interp(P->kappa + ((size_t)n * ng + g) * P->nT, P->T0, P->dT, P->nT, Tm);
      s += wg[g];
    }
    wn[n] = B_at(P, n, Tm) * s;
    if (orc_quantize(wg, ng, cg + (size_t)n * ng) != 0) {
      for (int g = 0; g < ng; ++g) wg[g] = 1.0;
      rc = orc_quantize(wg, ng, cg + (size_t)n * ng);
    }
  }
  if (rc == 0) rc = orc_quantize(wn, nb, cn);
  free(wn);
  free(wg);
  return rc;
}

static int pick(const uint64_t *cum, int K, uint32_t u) {
  for (int k = 0; k < K; ++k)
    if ((uint64_t)u < cum[k]) return k;
  return K - 1;
}

static uint64_t count_of(const uint64_t *cum, int k) { return k == 0 ? cum[0] : cum[k] - cum[k - 1]; }

/* ---- multigrid (Section 4.3) ------------------------------------------------ */
/* Overlaid grids, each coarsened by 2 from the previous one: grid 0 is the
 * problem's own, grid l + 1 holds in each of its cells the mean T and x of the
 * 2x2x2 cells of grid l it covers (the coarse temperatures come from the fine
 * solution).  A grid is added while every dimension of the previous one is even
 * and halves to at least 3 cells, the paper's smallest 3^3 mesh. */
enum { ORC_MG_MAX = 16 };

typedef struct {
  int L; /* grids in use */
  int k; /* segments marched on a grid before falling onto the next */
  int N[ORC_MG_MAX][3];
  double delta[ORC_MG_MAX][3];
  const double *T[ORC_MG_MAX], *x[ORC_MG_MAX]; /* x NULL: x_ref everywhere */
  double *own[ORC_MG_MAX];                     /* coarse T and x storage */
} mg_grids;

/* y of face F of grid lev (stretched grids: every 2^lev-th face of grid 0) */
static double yface(const orc_problem *P, int lev, int F) { return P->yf[(size_t)F << lev]; }

int orc_mg_max_levels(int nx, int ny, int nz) {
  int n[3] = {nx, ny, nz}, L = 1;
  while (L < ORC_MG_MAX) {
    int ok = 1;
    for (int a = 0; a < 3; ++a)
      if (n[a] % 2 != 0 || n[a] / 2 < 3) ok = 0;
    if (!ok) break;
    for (int a = 0; a < 3; ++a) n[a] /= 2;
    ++L;
  }
  return L;
}

static void mg_free(mg_grids *M) {
  for (int l = 0; l < ORC_MG_MAX; ++l) free(M->own[l]);
  memset(M, 0, sizeof(*M));
}

/* mean of the 8 children of coarse cell (I, J, K), z outermost, x innermost;
 * on a stretched grid weighted by the children's heights w[0], w[1] (the
 * volume-weighted mean) */
static double mean8(const double *v, const int n[3], int I, int J, int K, const double *w) {
  double s = 0.0, ws = 0.0;
  for (int c = 0; c < 2; ++c)
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a) {
        const double f =
            v[(size_t)(2 * I + a) + (size_t)n[0] * ((size_t)(2 * J + b) + (size_t)n[1] * (2 * K + c))];
        if (w) {
          s += w[b] * f;
          ws += w[b];
        } else {
          s += f;
        }
      }
  return w ? s / ws : s * 0.125;
}

static int mg_build(const orc_problem *P, int L, int k, mg_grids *M) {
  memset(M, 0, sizeof(*M));
  if (L < 1 || L > orc_mg_max_levels(P->nx, P->ny, P->nz) || k < 1) return -3;
  M->L = L;
  M->k = k;
  M->N[0][0] = P->nx;
  M->N[0][1] = P->ny;
  M->N[0][2] = P->nz;
  M->delta[0][0] = P->lx / P->nx;
  M->delta[0][1] = P->ly / P->ny;
  M->delta[0][2] = P->lz / P->nz;
  M->T[0] = P->T;
  M->x[0] = P->xh2o;
  for (int l = 1; l < L; ++l) {
    for (int a = 0; a < 3; ++a) M->N[l][a] = M->N[l - 1][a] / 2;
    M->delta[l][0] = P->lx / M->N[l][0];
    M->delta[l][1] = P->ly / M->N[l][1];
    M->delta[l][2] = P->lz / M->N[l][2];
    const size_t nc = (size_t)M->N[l][0] * M->N[l][1] * M->N[l][2];
    M->own[l] = (double *)malloc(sizeof(double) * nc * 2);
    if (!M->own[l]) {
      mg_free(M);
      return -4;
    }
    double *T = M->own[l], *x = P->xh2o ? M->own[l] + nc : NULL;
    for (int K = 0; K < M->N[l][2]; ++K)
      for (int J = 0; J < M->N[l][1]; ++J)
        for (int I = 0; I < M->N[l][0]; ++I) {
          const size_t c = (size_t)I + (size_t)M->N[l][0] * ((size_t)J + (size_t)M->N[l][1] * K);
          double wy[2];
          if (P->yf) {
            wy[0] = yface(P, l - 1, 2 * J + 1) - yface(P, l - 1, 2 * J);
            wy[1] = yface(P, l - 1, 2 * J + 2) - yface(P, l - 1, 2 * J + 1);
          }
          T[c] = mean8(M->T[l - 1], M->N[l - 1], I, J, K, P->yf ? wy : NULL);
          if (x) x[c] = mean8(M->x[l - 1], M->N[l - 1], I, J, K, P->yf ? wy : NULL);
        }
    M->T[l] = T;
    M->x[l] = x;
  }
  return 0;
}

/* ---- one ray: Algorithm 1 "March", Eqs. 2, 3, 14 ---------------------------- */

typedef struct {
  double *row; /* per-ray exchange kappa_i tau alpha_j per cell j, or NULL */
  unsigned char *mark;
  int *touched;
  int ntouched;
  double wall[2];
  long last;   /* the last medium cell the ray crossed (linear index) */
  double res;  /* kappa_i tau at termination: the residual absorbed there */
} xch_acc;

static void trace_core(const orc_problem *P, const mg_grids *M, int n, int g, const int cell0[3],
                       const double frac0[3], const double dir0[3], double tol,
                       int max_steps, uint64_t seed, uint32_t cellid, uint32_t ray,
                       uint32_t snap, orc_ray_out *o, xch_acc *xa) {
  int N[3] = {P->nx, P->ny, P->nz};
  double delta[3] = {P->lx / P->nx, P->ly / P->ny, P->lz / P->nz};
  const double *Tl = P->T, *xl = P->xh2o; /* fields of the current grid */
  int lev = 0, lsteps = 0;                /* current grid, segments marched on it */
  int c[3] = {cell0[0], cell0[1], cell0[2]};
  double fr[3] = {frac0[0], frac0[1], frac0[2]};
  double d[3] = {dir0[0], dir0[1], dir0[2]};

  const size_t ci = (size_t)c[0] + (size_t)N[0] * ((size_t)c[1] + (size_t)N[1] * c[2]);
  const double kap_i = kappa_at(P, n, g, P->T[ci], x_of(P, ci));
  const double B_i = B_at(P, n, P->T[ci]);

  double X = 0.0, absX = 0.0, Xw = 0.0, tau = 1.0, path = 0.0, B_last = B_i;
  size_t j_last = ci;
  int64_t steps = 0;
  int capped = 0, walls = 0;
  uint32_t nrefl = 0;

  /* Parametric ray o + t d: the m-th crossing of an axis-a face happens at
   * t = (g0_a + m) * tstep_a with g0_a the distance to the first face in units of
   * the cell size along the ray (Algorithm 1: df = dp / dir). */
  double g0[3], tstep[3], tnext[3];
  int sgn[3];
  int64_t cnt[3];
  double tprev;
  /* stretched y: the crossing of face F is at t = (y_F - y_o) / d_y, with y_o
   * the y of the current straight piece's start */
  const int sy = P->yf != NULL;
  double y_o = 0.0;
restart:
  for (int a = 0; a < 3; ++a) {
    cnt[a] = 0;
    if (d[a] > 0.0) {
      sgn[a] = 1;
      g0[a] = 1.0 - fr[a];
    } else if (d[a] < 0.0) {
      sgn[a] = -1;
      g0[a] = fr[a];
    } else {
      sgn[a] = 0;
      g0[a] = 0.0;
    }
    tstep[a] = sgn[a] ? delta[a] / fabs(d[a]) : INFINITY;
    tnext[a] = sgn[a] ? g0[a] * tstep[a] : INFINITY;
  }
  if (sy) {
    const double y0 = yface(P, lev, c[1]), y1 = yface(P, lev, c[1] + 1);
    y_o = y0 + fr[1] * (y1 - y0);
    if (sgn[1] > 0) tnext[1] = (y1 - y_o) / d[1];
    if (sgn[1] < 0) tnext[1] = (y0 - y_o) / d[1];
  }
  tprev = 0.0;

  for (;;) {
    if (M && lev + 1 < M->L && lsteps >= M->k) {
      /* multigrid (Section 4.3): after k segments on this grid the ray falls onto
       * the next coarser one at its current point; its position inside the
       * coarse cell follows from the position inside the current cell */
      for (int b = 0; b < 3; ++b) {
        if (sy && b == 1) {
          /* stretched y: the current y within the coarse cell's faces */
          const double yc = y_o + tprev * d[1];
          const double y0 = yface(P, lev + 1, c[1] >> 1), y1 = yface(P, lev + 1, (c[1] >> 1) + 1);
          fr[1] = (yc - y0) / (y1 - y0);
          if (fr[1] < 0.0) fr[1] = 0.0;
          if (fr[1] > 1.0) fr[1] = 1.0;
          c[1] >>= 1;
          continue;
        }
        if (sgn[b] > 0)
          fr[b] = 1.0 - (tnext[b] - tprev) / tstep[b];
        else if (sgn[b] < 0)
          fr[b] = (tnext[b] - tprev) / tstep[b];
        if (fr[b] < 0.0) fr[b] = 0.0;
        if (fr[b] > 1.0) fr[b] = 1.0;
        fr[b] = ((double)(c[b] & 1) + fr[b]) * 0.5;
        c[b] >>= 1;
      }
      ++lev;
      lsteps = 0;
      for (int b = 0; b < 3; ++b) {
        N[b] = M->N[lev][b];
        delta[b] = M->delta[lev][b];
      }
      Tl = M->T[lev];
      xl = M->x[lev];
      goto restart;
    }
    int a = 0; /* face crossed first; lowest axis on ties */
    if (tnext[1] < tnext[a]) a = 1;
    if (tnext[2] < tnext[a]) a = 2;
    double ds = tnext[a] - tprev;
    if (ds < 0.0) ds = 0.0;
    const size_t j = (size_t)c[0] + (size_t)N[0] * ((size_t)c[1] + (size_t)N[1] * c[2]);
    const double kap_j = kappa_at(P, n, g, Tl[j], xl ? xl[j] : P->x_ref);
    const double B_j = B_at(P, n, Tl[j]);
    const double alpha = -expm1(-kap_j * ds); /* Eq. 2: 1 - exp(-kappa_j l_j) */
    const double term = kap_i * (B_i - B_j) * tau * alpha; /* Eq. 14 per segment */
    if (xa && xa->row) {
      if (!xa->mark[j]) {
        xa->mark[j] = 1;
        xa->touched[xa->ntouched++] = (int)j;
      }
      xa->row[j] += kap_i * tau * alpha;
    }
    X += term;
    absX += fabs(term);
    tau *= exp(-kap_j * ds); /* Eq. 3: tau *= (1 - alpha) */
    B_last = B_j;
    j_last = j;
    path += ds;
    ++steps;
    ++lsteps;
    if (tau <= tol) break;
    if (steps >= max_steps) {
      capped = 1;
      break;
    }
    /* step into the neighbour across face a */
    tprev = tnext[a];
    ++cnt[a];
    tnext[a] = (g0[a] + (double)cnt[a]) * tstep[a];
    c[a] += sgn[a];
    if (sy && a == 1 && c[1] >= 0 && c[1] < N[1])
      tnext[1] = (yface(P, lev, c[1] + (sgn[1] > 0)) - y_o) / d[1];
    if (P->xz_walls && a != 1 && (c[a] < 0 || c[a] >= N[a])) {
      /* closed box: a black wall at an x or z face absorbs what is left and
       * emits at its temperature (Eq. 3 wall factor with eps = 1) */
      const int f = (a == 0 ? 0 : 2) + (c[a] < 0 ? 0 : 1);
      const double B_w = B_at(P, n, P->T_xz[f]);
      const double tw = kap_i * (B_i - B_w) * tau;
      X += tw;
      absX += fabs(tw);
      Xw += tw;
      ++walls;
      tau = 0.0;
      break;
    }
    if (a == 0) c[0] = (c[0] % N[0] + N[0]) % N[0]; /* periodic x */
    if (a == 2) c[2] = (c[2] % N[2] + N[2]) % N[2]; /* periodic z */
    if (a == 1 && (c[1] < 0 || c[1] >= N[1])) {
      const int w = c[1] < 0 ? 0 : 1;
      const double eps = P->eps_wall[w];
      const double B_w = B_at(P, n, P->T_wall[w]);
      const double tw = kap_i * (B_i - B_w) * tau * eps; /* wall as absorber j */
      if (xa) xa->wall[w] += kap_i * tau * eps;
      X += tw;
      absX += fabs(tw);
      Xw += tw;
      ++walls;
      tau *= (1.0 - eps); /* Eq. 3, wall factor */
      if (eps >= 1.0 || tau <= tol) break;
      /* reflect from the crossing point */
      for (int b = 0; b < 3; ++b) {
        if (b == 1) continue;
        if (sgn[b] > 0)
          fr[b] = 1.0 - (tnext[b] - tprev) / tstep[b];
        else if (sgn[b] < 0)
          fr[b] = (tnext[b] - tprev) / tstep[b];
        /* no motion along b: the fraction is unchanged */
        if (fr[b] < 0.0) fr[b] = 0.0;
        if (fr[b] > 1.0) fr[b] = 1.0;
      }
      c[1] = (w == 0) ? 0 : N[1] - 1;
      fr[1] = (w == 0) ? 0.0 : 1.0;
      if (P->reflect == 1) {
        d[1] = -d[1];
      } else {
        uint32_t u[4];
        draw(seed, cellid, ray, 2u + nrefl, snap, u);
        const double mu = sqrt(orc_uniform(u[0])); /* Lambertian: cos = sqrt(U) */
        const double phi = 2.0 * M_PI * orc_uniform(u[1]);
        const double s = sqrt(fmax(0.0, 1.0 - mu * mu));
        d[0] = s * cos(phi);
        d[1] = (w == 0) ? mu : -mu;
        d[2] = s * sin(phi);
      }
      ++nrefl;
      goto restart;
    }
  }
  /* residual dump into the emitting cell (Algorithm 1) */
  if (tau > 0.0) {
    const double tr = kap_i * (B_i - B_last) * tau;
    X += tr;
    absX += fabs(tr);
  }
  if (xa) {
    xa->last = (long)j_last;
    xa->res = tau > 0.0 ? kap_i * tau : 0.0;
  }
  o->X = X;
  o->abs_terms = absX;
  o->X_wall = Xw;
  o->tau_end = tau;
  o->steps = steps;
  o->capped = capped;
  o->walls = walls;
  o->path = path;
}

int orc_trace_ray(const orc_problem *P, const orc_ray_in *in, orc_ray_out *out) {
  if (in->n < 0 || in->n >= P->n_bands || in->g < 0 || in->g >= P->n_g) return -1;
  const uint32_t cellid =
      (uint32_t)(in->cell[0] + P->nx * (in->cell[1] + P->ny * in->cell[2]));
  trace_core(P, NULL, in->n, in->g, in->cell, in->frac, in->dir, in->tol, in->max_steps, in->seed,
             cellid, in->ray, in->snapshot, out, NULL);
  return 0;
}

int orc_trace_ray_mg(const orc_problem *P, const orc_ray_in *in, int mg_levels, int mg_steps,
                     orc_ray_out *out) {
  if (in->n < 0 || in->n >= P->n_bands || in->g < 0 || in->g >= P->n_g) return -1;
  mg_grids M;
  const int rc = mg_build(P, mg_levels < 1 ? 1 : mg_levels, mg_steps, &M);
  if (rc != 0) return rc;
  const uint32_t cellid =
      (uint32_t)(in->cell[0] + P->nx * (in->cell[1] + P->ny * in->cell[2]));
  trace_core(P, &M, in->n, in->g, in->cell, in->frac, in->dir, in->tol, in->max_steps, in->seed,
             cellid, in->ray, in->snapshot, out, NULL);
  mg_free(&M);
  return 0;
}

/* ---- one ray's sampled state (Algorithm 1 "Initialize", Eqs. 9, 16, 17) ----- */

typedef struct {
  int n, g;
  int h;           /* 0: upward hemisphere (d_y > 0), 1: downward */
  double p_ng;     /* p(n,g) the ray was drawn with */
  double p_h;      /* probability of its hemisphere */
  double w;        /* w_g / (p(n,g) q(Omega)) */
  double frac[3];
  double dir[3];
} ray_init;

static void init_ray(const orc_problem *P, const orc_params *S, const uint64_t *cn,
                     const uint64_t *cg, uint32_t hemi, uint32_t cellid, uint32_t ray,
                     ray_init *R) {
  uint32_t u[4];
  draw(S->seed, cellid, ray, 0u, S->snapshot, u);
  /* polar direction (Eq. 9 with the y axis as pole): upward hemisphere when the
   * top 23 bits of R_theta fall below the count `hemi` of 2^23, mu uniform inside
   * the chosen hemisphere; hemi = 2^22 gives mu = 1 - 2 U(R_theta) exactly */
  const uint32_t m0 = u[0] >> 9;
  double mu, ph;
  if (m0 < hemi) {
    mu = 1.0 - ((double)m0 + 0.5) / (double)hemi;
    ph = (double)hemi * 0x1p-23;
    R->h = 0;
  } else {
    mu = -(((double)(m0 - hemi)) + 0.5) / (double)(8388608u - hemi);
    ph = (double)(8388608u - hemi) * 0x1p-23;
    R->h = 1;
  }
  R->p_h = ph;
  const double phi = 2.0 * M_PI * orc_uniform(u[1]);
  const double s = sqrt(fmax(0.0, 1.0 - mu * mu));
  R->dir[0] = s * cos(phi);
  R->dir[1] = mu;
  R->dir[2] = s * sin(phi);
  /* band n from R_n = u[2], quadrature point g from R_g = u[3] (Eq. 17) */
  const int nb = P->n_bands, ng = P->n_g;
  R->n = pick(cn, nb, u[2]);
  R->g = pick(cg + (size_t)R->n * ng, ng, u[3]);
  const double p = ((double)count_of(cn, R->n) * 0x1p-32) *
                   ((double)count_of(cg + (size_t)R->n * ng, R->g) * 0x1p-32);
  R->p_ng = p;
  R->w = (P->w_g[R->g] / p) * (2.0 * M_PI / ph);
  if (S->origin == 1) {
    R->frac[0] = R->frac[1] = R->frac[2] = 0.5;
  } else {
    uint32_t v[4];
    draw(S->seed, cellid, ray, 1u, S->snapshot, v);
    R->frac[0] = orc_uniform(v[0]);
    R->frac[1] = orc_uniform(v[1]);
    R->frac[2] = orc_uniform(v[2]);
  }
}

/* ---- solve over a box of emitting cells ------------------------------------ */

typedef struct {
  const orc_problem *P;
  const orc_params *S;
  orc_cell_sums *out;
  const uint64_t *cn, *cg;
  int bi0, bj0, bk0, bnx, bny, bnz;
  atomic_long next;
  long total;
  /* exchange mode */
  double *G, *G2, *Gw, *Gw2;
  pthread_mutex_t lock;
  const mg_grids *M; /* multigrid, or NULL */
} solve_job;

static void solve_cell(solve_job *J, long b, xch_acc *xa) {
  const orc_problem *P = J->P;
  const orc_params *S = J->S;
  const int i = J->bi0 + (int)(b % J->bnx);
  const int j = J->bj0 + (int)((b / J->bnx) % J->bny);
  const int k = J->bk0 + (int)(b / ((long)J->bnx * J->bny));
  const uint32_t cellid = (uint32_t)(i + P->nx * (j + P->ny * k));
  const int nb = P->n_bands, ng = P->n_g;
  const uint64_t *cn = S->cell_cn ? S->cell_cn + (size_t)b * nb : J->cn;
  const uint64_t *cg = S->cell_cg ? S->cell_cg + (size_t)b * nb * ng : J->cg;
  const uint32_t hemi = S->cell_hemi ? S->cell_hemi[b] : 4194304u;
  double sy = 0, sy2 = 0, sa = 0, sw = 0, sw2 = 0;
  uint64_t st = 0, cap = 0;
  const int cell0[3] = {i, j, k};
  for (int r = 0; r < S->rays_per_cell; ++r) {
    const uint32_t ray = (uint32_t)(S->ray_offset + (uint64_t)r);
    ray_init R;
    init_ray(P, S, cn, cg, hemi, cellid, ray, &R);
    orc_ray_out o;
    if (xa) {
      xa->ntouched = 0;
      xa->wall[0] = xa->wall[1] = 0.0;
    }
    trace_core(P, J->M, R.n, R.g, cell0, R.frac, R.dir, S->tol, S->max_steps, S->seed, cellid,
               ray, S->snapshot, &o, xa);
    const double Y = R.w * o.X;
    const size_t tix = (size_t)b * nb * ng * 2 + ((size_t)R.n * ng + R.g) * 2 + R.h;
    if (S->tally) S->tally[tix] += Y * Y * R.p_ng * R.p_h / (double)S->rays_per_cell;
    if (S->tally_cost)
      S->tally_cost[tix] += (double)o.steps / (R.p_ng * R.p_h) / (double)S->rays_per_cell;
    sy += Y;
    sy2 += Y * Y;
    sa += R.w * o.abs_terms;
    sw += R.w * o.X_wall;
    sw2 += (R.w * o.X_wall) * (R.w * o.X_wall);
    st += (uint64_t)o.steps;
    cap += (uint64_t)o.capped;
    if (xa) {
      const size_t nc = (size_t)P->nx * P->ny * P->nz;
      for (int t = 0; t < xa->ntouched; ++t) {
        const int jj = xa->touched[t];
        const double v = R.w * xa->row[jj];
        J->G[(size_t)cellid * nc + jj] += v;
        J->G2[(size_t)cellid * nc + jj] += v * v;
        xa->row[jj] = 0.0;
        xa->mark[jj] = 0;
      }
      for (int w = 0; w < 2; ++w) {
        const double v = R.w * xa->wall[w];
        J->Gw[(size_t)cellid * 2 + w] += v;
        J->Gw2[(size_t)cellid * 2 + w] += v * v;
      }
    }
  }
  if (J->out) {
    J->out->sum_y[b] = sy;
    J->out->sum_y2[b] = sy2;
    J->out->sum_abs[b] = sa;
    J->out->sum_wall[b] = sw;
    J->out->sum_wall2[b] = sw2;
    J->out->steps[b] = st;
    J->out->capped[b] = cap;
  }
}

static void *solve_worker(void *arg) {
  solve_job *J = (solve_job *)arg;
  xch_acc xa, *pxa = NULL;
  if (J->G) {
    const size_t nc = (size_t)J->P->nx * J->P->ny * J->P->nz;
    xa.row = (double *)calloc(nc, sizeof(double));
    xa.mark = (unsigned char *)calloc(nc, 1);
    xa.touched = (int *)malloc(sizeof(int) * nc);
    pxa = &xa;
  }
  for (;;) {
    const long b = atomic_fetch_add(&J->next, 1);
    if (b >= J->total) break;
    solve_cell(J, b, pxa);
  }
  if (pxa) {
    free(xa.row);
    free(xa.mark);
    free(xa.touched);
  }
  return NULL;
}

static int run_jobs(solve_job *J, int nthreads) {
  if (nthreads <= 1 || J->total <= 1) {
    solve_worker(J);
    return 0;
  }
  if (nthreads > 256) nthreads = 256;
  pthread_t th[256];
  int started = 0;
  for (int t = 0; t < nthreads; ++t)
    if (pthread_create(&th[t], NULL, solve_worker, J) == 0) ++started;
  if (started == 0) solve_worker(J);
  for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
  return 0;
}

static int setup_job(const orc_problem *P, const orc_params *S, solve_job *J, uint64_t *cn,
                     uint64_t *cg) {
  memset(J, 0, sizeof(*J));
  J->P = P;
  J->S = S;
  int b[6] = {0, P->nx, 0, P->ny, 0, P->nz};
  if (S->use_box) memcpy(b, S->box, sizeof(b));
  if (b[0] < 0 || b[1] > P->nx || b[2] < 0 || b[3] > P->ny || b[4] < 0 || b[5] > P->nz)
    return -1;
  J->bi0 = b[0];
  J->bj0 = b[2];
  J->bk0 = b[4];
  J->bnx = b[1] > b[0] ? b[1] - b[0] : 0;
  J->bny = b[3] > b[2] ? b[3] - b[2] : 0;
  J->bnz = b[5] > b[4] ? b[5] - b[4] : 0;
  J->total = (long)J->bnx * J->bny * J->bnz;
  atomic_init(&J->next, 0);
  if (orc_plain_proposal(P, cn, cg, NULL) != 0) return -2;
  J->cn = cn;
  J->cg = cg;
  return 0;
}

int orc_solve(const orc_problem *P, const orc_params *S, orc_cell_sums *out) {
  uint64_t *cn = (uint64_t *)malloc(sizeof(uint64_t) * P->n_bands);
  uint64_t *cg = (uint64_t *)malloc(sizeof(uint64_t) * P->n_bands * P->n_g);
  solve_job J;
  mg_grids M;
  int use_mg = S->mg_levels > 1;
  int rc = use_mg ? mg_build(P, S->mg_levels, S->mg_steps, &M) : 0;
  if (rc == 0) rc = setup_job(P, S, &J, cn, cg);
  if (rc == 0) {
    J.out = out;
    J.M = use_mg ? &M : NULL;
    run_jobs(&J, S->nthreads);
  }
  if (use_mg) mg_free(&M);
  free(cn);
  free(cg);
  return rc;
}

/* Exchange tallies for the reciprocity check (Eq. 11): G[i][j] sums, over rays
 * leaving cell i, w kappa_i tau alpha_j; Gw[i][w] the same for the walls.  Whole
 * grid only; runs single-threaded so that the sums need no locking. */
int orc_exchange(const orc_problem *P, const orc_params *S, double *G, double *G2, double *Gw,
                 double *Gw2) {
  uint64_t *cn = (uint64_t *)malloc(sizeof(uint64_t) * P->n_bands);
  uint64_t *cg = (uint64_t *)malloc(sizeof(uint64_t) * P->n_bands * P->n_g);
  orc_params S2 = *S;
  S2.use_box = 0;
  S2.cell_cn = NULL;
  S2.cell_cg = NULL;
  S2.cell_hemi = NULL;
  solve_job J;
  int rc = setup_job(P, &S2, &J, cn, cg);
  if (rc == 0) {
    J.G = G;
    J.G2 = G2;
    J.Gw = Gw;
    J.Gw2 = Gw2;
    run_jobs(&J, 1);
  }
  free(cn);
  free(cg);
  return rc;
}

/* ---- deterministic quadrature of the same estimand ------------------------- */
/* Q_i = sum_{n,g} w_g (1/V_i) int_{V_i} int_{4pi} X dOmega dV with a tensor rule:
 * mu nodes/weights on [-1, 1], nphi midpoints in phi, and over the cell either
 * a tensor rule, an explicit list of origins (origin 0) or the centre (origin 1).  Needs black or specular walls
 * (diffuse reflection would need random draws). */
typedef struct {
  const orc_problem *P;
  const double *mu, *mu_w, *vn, *vw;
  int nmu, nphi, nv, origin, max_steps;
  double tol;
  const int *cells;
  double *q;
  atomic_long next;
  long total;
} quad_job;

static void *quad_worker(void *arg) {
  quad_job *Q = (quad_job *)arg;
  const orc_problem *P = Q->P;
  for (;;) {
    const long t = atomic_fetch_add(&Q->next, 1);
    if (t >= Q->total) break;
    const int c = Q->cells[t];
    const int cell0[3] = {c % P->nx, (c / P->nx) % P->ny, c / (P->nx * P->ny)};
    double acc = 0.0;
    /* origins: the centre, an nv^3 tensor rule (nv > 0) or an explicit list of
     * -nv fractions (x,y,z) with weights (nv < 0) */
    const int nvol = Q->origin == 1 ? 1 : (Q->nv > 0 ? Q->nv * Q->nv * Q->nv : -Q->nv);
    for (int n = 0; n < P->n_bands; ++n)
      for (int g = 0; g < P->n_g; ++g)
        for (int im = 0; im < Q->nmu; ++im)
          for (int ip = 0; ip < Q->nphi; ++ip) {
            const double mu = Q->mu[im];
            const double phi = 2.0 * M_PI * ((double)ip + 0.5) / (double)Q->nphi;
            const double s = sqrt(fmax(0.0, 1.0 - mu * mu));
            const double dir[3] = {s * cos(phi), mu, s * sin(phi)};
            const double wa = P->w_g[g] * Q->mu_w[im] * (2.0 * M_PI / (double)Q->nphi);
            for (int v = 0; v < nvol; ++v) {
              double fr[3] = {0.5, 0.5, 0.5};
              double wv = 1.0;
              if (Q->origin != 1 && Q->nv > 0) {
                const int a = v % Q->nv, b = (v / Q->nv) % Q->nv, e = v / (Q->nv * Q->nv);
                fr[0] = Q->vn[a];
                fr[1] = Q->vn[b];
                fr[2] = Q->vn[e];
                wv = Q->vw[a] * Q->vw[b] * Q->vw[e];
              } else if (Q->origin != 1) {
                fr[0] = Q->vn[3 * v];
                fr[1] = Q->vn[3 * v + 1];
                fr[2] = Q->vn[3 * v + 2];
                wv = Q->vw[v];
              }
              orc_ray_out o;
              trace_core(P, NULL, n, g, cell0, fr, dir, Q->tol, Q->max_steps, 0, (uint32_t)c, 0, 0, &o,
                         NULL);
              acc += wa * wv * o.X;
            }
          }
    Q->q[t] = acc;
  }
  return NULL;
}

int orc_quadrature(const orc_problem *P, const double *mu, const double *mu_w, int nmu,
                   int nphi, const double *vn, const double *vw, int nv, int origin,
                   double tol, int max_steps, const int *cells, int ncq, int nthreads,
                   double *q) {
  for (int w = 0; w < 2; ++w)
    if (P->eps_wall[w] < 1.0 && P->reflect != 1) return -1;
  quad_job Q;
  memset(&Q, 0, sizeof(Q));
  Q.P = P;
  Q.mu = mu;
  Q.mu_w = mu_w;
  Q.vn = vn;
  Q.vw = vw;
  Q.nmu = nmu;
  Q.nphi = nphi;
  Q.nv = nv;
  Q.origin = origin;
  Q.tol = tol;
  Q.max_steps = max_steps;
  Q.cells = cells;
  Q.q = q;
  Q.total = ncq;
  atomic_init(&Q.next, 0);
  if (nthreads <= 1) {
    quad_worker(&Q);
    return 0;
  }
  if (nthreads > 256) nthreads = 256;
  pthread_t th[256];
  int started = 0;
  for (int t = 0; t < nthreads; ++t)
    if (pthread_create(&th[t], NULL, quad_worker, &Q) == 0) ++started;
  if (started == 0) quad_worker(&Q);
  for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
  return 0;
}

/* ---- absorption-based reciprocal estimate (ARMC) -----------------------------
 * Eq. FM writes Q^R_i as the power cell i emits minus the power it absorbs;
 * with the reciprocity relation (Q_(i->j),nu / I_b,nu(T_i) = Q_(j->i),nu /
 * I_b,nu(T_j)) every exchange can be estimated from the rays of either cell.
 * The emission-based estimate (orc_solve) takes cell i's exchanges from cell i's
 * own rays.  This absorption-based one takes cell i's exchange with every other
 * medium cell j from the rays EMITTED BY j that are absorbed in i: a ray of cell
 * j with weight w deposits, for each cell i it crosses,
 *     (V_j / V_i) w kappa_j (B_i - B_j) tau alpha_i
 * (minus the term it adds to cell j's emission-based estimate, moved to the cell
 * that absorbs), and its residual kappa_j (B_last - B_j) tau in the last cell it
 * crossed (the cut-off convention of Algorithm 1, from the other side).  The
 * exchange with the walls stays estimated from cell i's own rays (the walls emit
 * no rays here).  Every cell of the grid emits; the sums are split into K batches
 * by ray index (r mod K) for a batch-means standard error.
 *   acc [K][nc]: sum over rays of the batch of the deposits into each cell;
 *   absacc [nc]: sum of |deposits| (the parity scale);
 *   accE [K][nc] (nullable): the emission-based sums of each cell's own samples
 *   per batch (for the combination of the two estimates);
 *   steps [nc]: medium segments of each cell's own rays.
 * Single grid only (no multigrid); threads take fixed ranges of emitting cells
 * and their partial sums are added in thread order, so the result is
 * deterministic. */

typedef struct {
  const orc_problem *P;
  const orc_params *S;
  const uint64_t *cn, *cg;
  long c0, c1;
  int K;
  double *acc, *absacc, *accE;
  uint64_t *steps;
} armc_job;

static double cell_volume(const orc_problem *P, long c) {
  const int j = (int)((c / P->nx) % P->ny);
  const double dy = P->yf ? P->yf[j + 1] - P->yf[j] : P->ly / P->ny;
  return (P->lx / P->nx) * dy * (P->lz / P->nz);
}

static void *armc_worker(void *arg) {
  armc_job *J = (armc_job *)arg;
  const orc_problem *P = J->P;
  const orc_params *S = J->S;
  const size_t nc = (size_t)P->nx * P->ny * P->nz;
  const int nb = P->n_bands, ng = P->n_g;
  xch_acc xa;
  xa.row = (double *)calloc(nc, sizeof(double));
  xa.mark = (unsigned char *)calloc(nc, 1);
  xa.touched = (int *)malloc(sizeof(int) * nc);
  for (long c = J->c0; c < J->c1; ++c) {
    const int cell0[3] = {(int)(c % P->nx), (int)((c / P->nx) % P->ny), (int)(c / ((long)P->nx * P->ny))};
    const uint64_t *cn = S->cell_cn ? S->cell_cn + (size_t)c * nb : J->cn;
    const uint64_t *cg = S->cell_cg ? S->cell_cg + (size_t)c * nb * ng : J->cg;
    const uint32_t hemi = S->cell_hemi ? S->cell_hemi[c] : 4194304u;
    const double Vc = cell_volume(P, c);
    for (int r = 0; r < S->rays_per_cell; ++r) {
      const uint32_t ray = (uint32_t)(S->ray_offset + (uint64_t)r);
      ray_init R;
      init_ray(P, S, cn, cg, hemi, (uint32_t)c, ray, &R);
      orc_ray_out o;
      xa.ntouched = 0;
      xa.wall[0] = xa.wall[1] = 0.0;
      trace_core(P, NULL, R.n, R.g, cell0, R.frac, R.dir, S->tol, S->max_steps, S->seed, (uint32_t)c,
                 ray, S->snapshot, &o, &xa);
      double *accb = J->acc + (size_t)(r % J->K) * nc;
      const double B_e = B_at(P, R.n, P->T[c]);
      for (int t = 0; t < xa.ntouched; ++t) {
        const int jj = xa.touched[t];
        const double d = R.w * (B_at(P, R.n, P->T[jj]) - B_e) * xa.row[jj] * (Vc / cell_volume(P, jj));
        accb[jj] += d;
        J->absacc[jj] += fabs(d);
        xa.row[jj] = 0.0;
        xa.mark[jj] = 0;
      }
      if (xa.res != 0.0) {
        const double d = R.w * (B_at(P, R.n, P->T[xa.last]) - B_e) * xa.res * (Vc / cell_volume(P, xa.last));
        accb[xa.last] += d;
        J->absacc[xa.last] += fabs(d);
      }
      const double dw = R.w * o.X_wall; /* the cell's own exchange with the walls */
      accb[c] += dw;
      J->absacc[c] += fabs(dw);
      if (J->accE) J->accE[(size_t)(r % J->K) * nc + c] += R.w * o.X;
      J->steps[c] += (uint64_t)o.steps;
    }
  }
  free(xa.row);
  free(xa.mark);
  free(xa.touched);
  return NULL;
}

int orc_solve_armc(const orc_problem *P, const orc_params *S, int K, double *acc, double *absacc,
                   double *accE, uint64_t *steps) {
  if (K < 1 || S->mg_levels > 1) return -3;
  uint64_t *cn = (uint64_t *)malloc(sizeof(uint64_t) * P->n_bands);
  uint64_t *cg = (uint64_t *)malloc(sizeof(uint64_t) * P->n_bands * P->n_g);
  int rc = orc_plain_proposal(P, cn, cg, NULL);
  const long nc = (long)P->nx * P->ny * P->nz;
  int T = S->nthreads > 1 ? S->nthreads : 1;
  if (T > 256) T = 256;
  if (T > nc) T = (int)(nc > 0 ? nc : 1);
  armc_job *jobs = (armc_job *)calloc((size_t)T, sizeof(armc_job));
  if (rc == 0 && jobs) {
    for (int t = 0; t < T; ++t) {
      armc_job *J = &jobs[t];
      J->P = P;
      J->S = S;
      J->cn = cn;
      J->cg = cg;
      J->K = K;
      J->c0 = nc * t / T;
      J->c1 = nc * (t + 1) / T;
      J->acc = t ? (double *)calloc((size_t)K * nc, sizeof(double)) : acc;
      J->absacc = t ? (double *)calloc((size_t)nc, sizeof(double)) : absacc;
      J->accE = accE; /* each emitting cell belongs to one thread: no race */
      J->steps = steps;
    }
    pthread_t th[256];
    int started[256] = {0};
    for (int t = 1; t < T; ++t) {
      started[t] = pthread_create(&th[t], NULL, armc_worker, &jobs[t]) == 0;
      if (!started[t]) armc_worker(&jobs[t]);
    }
    armc_worker(&jobs[0]);
    for (int t = 1; t < T; ++t)
      if (started[t]) pthread_join(th[t], NULL);
    for (int t = 1; t < T; ++t) { /* thread order: deterministic sums */
      for (size_t q = 0; q < (size_t)K * nc; ++q) acc[q] += jobs[t].acc[q];
      for (long q = 0; q < nc; ++q) absacc[q] += jobs[t].absacc[q];
      free(jobs[t].acc);
      free(jobs[t].absacc);
    }
  } else if (rc == 0) {
    rc = -4;
  }
  free(jobs);
  free(cn);
  free(cg);
  return rc;
}
