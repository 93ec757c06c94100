/*
 * learn_oracle.c -- TEST INFRASTRUCTURE ONLY (not part of the product).
 *
 * Plain FP64 reference of the learned spectral/directional proposal.  The paper
 * samples (n, g) from Zhang's T_max pdf (Section 2.1, Eqs. 13 and 16) and the
 * direction isotropically (Eq. 9); any other pdf keeps Eq. 14 unbiased as long
 * as the ray weight divides by the probabilities actually used and every
 * (n, g, hemisphere) with a non-zero contribution keeps a non-zero probability.
 * The learned proposal replaces the pdf per emitting cell by
 *
 *   q(n,g) = (1 - mix) softmax(z)_(n,g) + mix p0(n,g)
 *   q(h)   = (1 - mix) softmax(z_up, z_down)_h + mix / 2
 *
 * with z the output of a 12 -> 64 -> 64 -> (K + 2) multilayer perceptron (GELU
 * activations) of local features of the cell and p0 the plain pdf.  Trained to
 * minimise, per emitting cell, the work to reach a given standard error --
 * second moment per ray times cost per ray -- relative to the plain proposal:
 *
 *   L_c = A(q) C(q) / (A(p0) C(p0)),   A(q) = sum_(k,h) m_c[k][h] / (q_k q_h),
 *                                      C(q) = c0 + sum_(k,h) c_c[k][h] q_k q_h,
 *
 * where m_c and c_c are the second-moment and cost tallies of a plain solve
 * (unbiased estimates of E[Y^2] and of the mean steps per ray under q) and c0
 * the fixed cost of a ray in steps.  Without cost tallies C = 1; the minimiser
 * of A alone over all pdfs is q proportional to sqrt(m).
 *
 * The batch form (mode 1) estimates the ratio of the GPU time a whole field
 * needs for a given relative error: with per-sample weights w_c = 1/ref_c^2
 * (ref_c the cell's error scale),
 *
 *   L = (sum_c w_c A_c(q) / sum_c w_c A_c(p0)) (sum_c C_c(q) / sum_c C_c(p0)):
 *
 * the mean relative second moment per ray times the mean cost per ray.
 *
 * Everything here is written from those definitions: no blocking or reordering
 * beyond the plain loops.  It shares no code with the CUDA library.
 */
#define _GNU_SOURCE
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "mcrt_oracle.h"

enum { F = ORC_NFEAT, H = ORC_HIDDEN };

/* ---- features of an emitting cell ------------------------------------------
 * 0 T_i / 1000            1 x_i                       2 y_c / h - 1
 * 3 T_wall,0 / 1000       4 T_wall,1 / 1000           5 eps of the nearer wall
 * 6 h dT/dy / 1000        7 h |grad_xz T| / 1000      8 mean T over 3^3 / T_i
 * 9 std T over 3^3 / T_i  10 kappa_P(T_i, x_i) h      11 T_max / T_i
 * (on a stretched grid y_c is the midpoint of the cell's faces and dT/dy divides
 * by the distance of the centres used)
 * with h = ly / 2 the channel half height, centred differences (one-sided at the
 * walls, periodic in x and z), the 3^3 neighbourhood periodic in x and z and cut
 * at the walls, and kappa_P the Planck mean of the tables at T_i:
 * sum_n B_n sum_g w_g kappa_(n,g) / sum_n B_n. */

static double T_at(const orc_problem *P, int i, int j, int k) {
  return P->T[(size_t)i + (size_t)P->nx * ((size_t)j + (size_t)P->ny * k)];
}

static int wrap(int i, int n) { return ((i % n) + n) % n; }

/* y of the centre of row j (stretched grids: midpoint of its faces) */
static double ycentre(const orc_problem *P, int j) {
  if (P->yf) return 0.5 * (P->yf[j] + P->yf[j + 1]);
  return (j + 0.5) * (P->ly / P->ny);
}

int orc_features(const orc_problem *P, const int32_t *cells, int64_t n, double T_max,
                 double *out) {
  const int nx = P->nx, ny = P->ny, nz = P->nz;
  const double dx = P->lx / nx, dy = P->ly / ny, dz = P->lz / nz, h = 0.5 * P->ly;
  const int nb = P->n_bands, ng = P->n_g, nT = P->nT;
  for (int64_t q = 0; q < n; ++q) {
    const int64_t c = cells[q];
    if (c < 0 || c >= (int64_t)nx * ny * nz) return -1;
    const int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / ((int64_t)nx * ny));
    const double Ti = P->T[c];
    const double xi = P->xh2o ? P->xh2o[c] : P->x_ref;
    const double yc = ycentre(P, j);
    double *f = out + q * F;
    f[0] = Ti / 1000.0;
    f[1] = xi;
    f[2] = yc / h - 1.0;
    f[3] = P->T_wall[0] / 1000.0;
    f[4] = P->T_wall[1] / 1000.0;
    f[5] = yc < h ? P->eps_wall[0] : P->eps_wall[1];
    double dTdy = 0.0;
    if (ny > 1 && !P->yf) {
      if (j == 0)
        dTdy = (T_at(P, i, 1, k) - T_at(P, i, 0, k)) / dy;
      else if (j == ny - 1)
        dTdy = (T_at(P, i, ny - 1, k) - T_at(P, i, ny - 2, k)) / dy;
      else
        dTdy = (T_at(P, i, j + 1, k) - T_at(P, i, j - 1, k)) / (2.0 * dy);
    } else if (ny > 1) {
      /* stretched grid: differences over the distances of the cell centres */
      const int j0 = j == 0 ? 0 : j - 1, j1 = j == ny - 1 ? ny - 1 : j + 1;
      dTdy = (T_at(P, i, j1, k) - T_at(P, i, j0, k)) / (ycentre(P, j1) - ycentre(P, j0));
    }
    f[6] = h * dTdy / 1000.0;
    const double dTdx = (T_at(P, wrap(i + 1, nx), j, k) - T_at(P, wrap(i - 1, nx), j, k)) / (2.0 * dx);
    const double dTdz = (T_at(P, i, j, wrap(k + 1, nz)) - T_at(P, i, j, wrap(k - 1, nz))) / (2.0 * dz);
    f[7] = h * sqrt(dTdx * dTdx + dTdz * dTdz) / 1000.0;
    double sum = 0.0;
    int cnt = 0;
    for (int c2 = -1; c2 <= 1; ++c2)
      for (int b2 = -1; b2 <= 1; ++b2)
        for (int a2 = -1; a2 <= 1; ++a2) {
          const int jj = j + b2;
          if (jj < 0 || jj >= ny) continue;
          sum += T_at(P, wrap(i + a2, nx), jj, wrap(k + c2, nz));
          ++cnt;
        }
    const double mean = sum / cnt;
    double var = 0.0;
    for (int c2 = -1; c2 <= 1; ++c2)
      for (int b2 = -1; b2 <= 1; ++b2)
        for (int a2 = -1; a2 <= 1; ++a2) {
          const int jj = j + b2;
          if (jj < 0 || jj >= ny) continue;
          const double d = T_at(P, wrap(i + a2, nx), jj, wrap(k + c2, nz)) - mean;
          var += d * d;
        }
    var /= cnt;
    f[8] = mean / Ti;
    f[9] = sqrt(var) / Ti;
    double num = 0.0, den = 0.0;
    for (int nn = 0; nn < nb; ++nn) {
      const double Bn = orc_interp(P->B + (size_t)nn * nT, P->T0, P->dT, nT, Ti);
      double s = 0.0;
      for (int g = 0; g < ng; ++g)
        s += P->w_g[g] * orc_interp(P->kappa + ((size_t)nn * ng + g) * nT, P->T0, P->dT, nT, Ti);
      num += Bn * s;
      den += Bn;
    }
    f[10] = den > 0.0 ? (num / den) * (xi / P->x_ref) * h : 0.0;
    f[11] = T_max / Ti;
  }
  return 0;
}

/* ---- the network ------------------------------------------------------------
 * theta = [W1 (H x F, row-major: output, input), b1 (H), W2 (H x H), b2 (H),
 *          W3 ((K + 2) x H), b3 (K + 2)].  Logits 0..K-1 are the spectral points
 * k = n n_g + g, logit K the upward and K + 1 the downward hemisphere. */

int64_t orc_mlp_nparams(int K) {
  return (int64_t)H * F + H + (int64_t)H * H + H + (int64_t)(K + 2) * H + (K + 2);
}

static double gelu(double x) { return 0.5 * x * (1.0 + erf(x / sqrt(2.0))); }

static double gelu_prime(double x) {
  return 0.5 * (1.0 + erf(x / sqrt(2.0))) + x * exp(-0.5 * x * x) / sqrt(2.0 * M_PI);
}

typedef struct {
  double xin[F], a1[H], h1[H], a2[H], h2[H];
  double *z, *s; /* [K + 2] */
} mlp_act;

static void forward_one(const double *theta, int K, const double *fmean, const double *finv,
                        const double *feat, mlp_act *A) {
  const double *W1 = theta, *b1 = W1 + H * F, *W2 = b1 + H, *b2 = W2 + H * H, *W3 = b2 + H,
               *b3 = W3 + (size_t)(K + 2) * H;
  for (int i = 0; i < F; ++i) A->xin[i] = (feat[i] - fmean[i]) * finv[i];
  for (int o = 0; o < H; ++o) {
    double a = b1[o];
    for (int i = 0; i < F; ++i) a += W1[o * F + i] * A->xin[i];
    A->a1[o] = a;
    A->h1[o] = gelu(a);
  }
  for (int o = 0; o < H; ++o) {
    double a = b2[o];
    for (int i = 0; i < H; ++i) a += W2[o * H + i] * A->h1[i];
    A->a2[o] = a;
    A->h2[o] = gelu(a);
  }
  for (int o = 0; o < K + 2; ++o) {
    double a = b3[o];
    for (int i = 0; i < H; ++i) a += W3[(size_t)o * H + i] * A->h2[i];
    A->z[o] = a;
  }
  /* softmax over the K spectral logits, and over the two hemisphere logits */
  double zmax = A->z[0];
  for (int k = 1; k < K; ++k) zmax = fmax(zmax, A->z[k]);
  double Z = 0.0;
  for (int k = 0; k < K; ++k) {
    A->s[k] = exp(A->z[k] - zmax);
    Z += A->s[k];
  }
  for (int k = 0; k < K; ++k) A->s[k] /= Z;
  const double hm = fmax(A->z[K], A->z[K + 1]);
  const double eu = exp(A->z[K] - hm), ed = exp(A->z[K + 1] - hm);
  A->s[K] = eu / (eu + ed);
  A->s[K + 1] = ed / (eu + ed);
}

static int act_alloc(mlp_act *A, int K) {
  A->z = (double *)malloc(sizeof(double) * (K + 2));
  A->s = (double *)malloc(sizeof(double) * (K + 2));
  return A->z && A->s ? 0 : -1;
}

static void act_free(mlp_act *A) {
  free(A->z);
  free(A->s);
}

int orc_mlp_forward(const double *theta, int K, const double *fmean, const double *finv,
                    const double *feat, int64_t n, const double *p0, int p0_stride, double mix,
                    double *q) {
  mlp_act A;
  if (K < 1 || act_alloc(&A, K) != 0) return -1;
  for (int64_t c = 0; c < n; ++c) {
    forward_one(theta, K, fmean, finv, feat + c * F, &A);
    const double *pc = p0 + c * p0_stride;
    double *qc = q + c * (K + 2);
    for (int k = 0; k < K; ++k) qc[k] = (1.0 - mix) * A.s[k] + mix * pc[k];
    qc[K] = (1.0 - mix) * A.s[K] + mix * 0.5;
    qc[K + 1] = (1.0 - mix) * A.s[K + 1] + mix * 0.5;
  }
  act_free(&A);
  return 0;
}

/* Mean over the n samples of L_c and its gradient with respect to theta (the
 * chain rule written out layer by layer).  m, cst [n][K][2] (cst NULL: no cost
 * factor), p0 [n][K].  A sample whose plain second moment is zero contributes
 * nothing; terms with p0_k = 0 are left out (that spectral point is never drawn
 * by the plain proposal, so its tallies are zero). */
/* Per-sample A(q), A(p0), C(q), C(p0) of sample c and dL/dq via the multipliers
 * gA = dL/dA_c(q), gC = dL/dC_c(q) (chain rule through the mixtures and the two
 * softmaxes, then layer by layer); adds the parameter gradient to grad. */
static void sample_terms(const mlp_act *A, int K, const double *mc, const double *cc, double c0,
                         const double *pc, double mix, double *q, double *Aq, double *A0, double *Cq,
                         double *C0) {
  for (int k = 0; k < K; ++k) q[k] = (1.0 - mix) * A->s[k] + mix * pc[k];
  q[K] = (1.0 - mix) * A->s[K] + mix * 0.5;
  q[K + 1] = (1.0 - mix) * A->s[K + 1] + mix * 0.5;
  *A0 = 0.0;
  *Aq = 0.0;
  *C0 = c0;
  *Cq = c0;
  for (int k = 0; k < K; ++k) {
    if (!(pc[k] > 0.0)) continue;
    for (int hh = 0; hh < 2; ++hh) {
      *A0 += mc[k * 2 + hh] / (pc[k] * 0.5);
      *Aq += mc[k * 2 + hh] / (q[k] * q[K + hh]);
      if (cc) {
        *C0 += cc[k * 2 + hh] * (pc[k] * 0.5);
        *Cq += cc[k * 2 + hh] * (q[k] * q[K + hh]);
      }
    }
  }
  if (!cc) *C0 = *Cq = 1.0;
}

static void sample_backward(const double *theta, int K, const mlp_act *A, const double *mc,
                            const double *cc, const double *pc, double mix, const double *q,
                            double gA, double gC, double *dz, double *gq, double *grad) {
  const double *W2 = theta + H * F + H, *W3 = W2 + H * H + H;
  double *gW1 = grad, *gb1 = gW1 + H * F, *gW2 = gb1 + H, *gb2 = gW2 + H * H, *gW3 = gb2 + H,
         *gb3 = gW3 + (size_t)(K + 2) * H;
  gq[K] = gq[K + 1] = 0.0;
  for (int k = 0; k < K; ++k) {
    gq[k] = 0.0;
    if (!(pc[k] > 0.0)) continue;
    for (int hh = 0; hh < 2; ++hh) {
      const double v = mc[k * 2 + hh];
      gq[k] -= gA * v / (q[k] * q[k] * q[K + hh]);
      gq[K + hh] -= gA * v / (q[k] * q[K + hh] * q[K + hh]);
      if (cc) {
        gq[k] += gC * cc[k * 2 + hh] * q[K + hh];
        gq[K + hh] += gC * cc[k * 2 + hh] * q[k];
      }
    }
  }
  double dot = 0.0;
  for (int k = 0; k < K; ++k) dot += A->s[k] * gq[k];
  for (int k = 0; k < K; ++k) dz[k] = (1.0 - mix) * A->s[k] * (gq[k] - dot);
  const double doth = A->s[K] * gq[K] + A->s[K + 1] * gq[K + 1];
  dz[K] = (1.0 - mix) * A->s[K] * (gq[K] - doth);
  dz[K + 1] = (1.0 - mix) * A->s[K + 1] * (gq[K + 1] - doth);
  double dh2[H], da2[H], dh1[H], da1[H];
  for (int i = 0; i < H; ++i) dh2[i] = 0.0;
  for (int o = 0; o < K + 2; ++o) {
    gb3[o] += dz[o];
    for (int i = 0; i < H; ++i) {
      gW3[(size_t)o * H + i] += dz[o] * A->h2[i];
      dh2[i] += W3[(size_t)o * H + i] * dz[o];
    }
  }
  for (int i = 0; i < H; ++i) da2[i] = dh2[i] * gelu_prime(A->a2[i]);
  for (int i = 0; i < H; ++i) dh1[i] = 0.0;
  for (int o = 0; o < H; ++o) {
    gb2[o] += da2[o];
    for (int i = 0; i < H; ++i) {
      gW2[o * H + i] += da2[o] * A->h1[i];
      dh1[i] += W2[o * H + i] * da2[o];
    }
  }
  for (int i = 0; i < H; ++i) da1[i] = dh1[i] * gelu_prime(A->a1[i]);
  for (int o = 0; o < H; ++o) {
    gb1[o] += da1[o];
    for (int i = 0; i < F; ++i) gW1[o * F + i] += da1[o] * A->xin[i];
  }
}

int orc_mlp_loss_grad(const double *theta, int K, const double *fmean, const double *finv,
                      const double *feat, const double *m, const double *cst, double c0,
                      const double *p0, const double *wgt, int mode, int64_t n, double mix,
                      double *loss, double *grad) {
  const int64_t np = orc_mlp_nparams(K);
  memset(grad, 0, sizeof(double) * np);
  *loss = 0.0;
  if (n <= 0) return 0;
  mlp_act A;
  if (K < 1 || act_alloc(&A, K) != 0) return -1;
  double *dz = (double *)malloc(sizeof(double) * (K + 2));
  double *gq = (double *)malloc(sizeof(double) * (K + 2));
  double *q = (double *)malloc(sizeof(double) * (K + 2));
  if (!dz || !gq || !q) {
    act_free(&A);
    free(dz);
    free(gq);
    free(q);
    return -1;
  }
  /* batch sums for mode 1 */
  double SAq = 0.0, SA0 = 0.0, SCq = 0.0, SC0 = 0.0;
  if (mode == 1) {
    for (int64_t c = 0; c < n; ++c) {
      forward_one(theta, K, fmean, finv, feat + c * F, &A);
      double Aq, A0, Cq, C0;
      sample_terms(&A, K, m + c * (int64_t)K * 2, cst ? cst + c * (int64_t)K * 2 : NULL, c0,
                   p0 + c * (int64_t)K, mix, q, &Aq, &A0, &Cq, &C0);
      const double w = wgt ? wgt[c] : 1.0;
      SAq += w * Aq;
      SA0 += w * A0;
      SCq += Cq;
      SC0 += C0;
    }
    if (!(SA0 > 0.0) || !(SC0 > 0.0)) goto done;
    *loss = (SAq / SA0) * (SCq / SC0);
  }
  for (int64_t c = 0; c < n; ++c) {
    forward_one(theta, K, fmean, finv, feat + c * F, &A);
    const double *mc = m + c * (int64_t)K * 2, *pc = p0 + c * (int64_t)K;
    const double *cc = cst ? cst + c * (int64_t)K * 2 : NULL;
    double Aq, A0, Cq, C0, gA, gC;
    sample_terms(&A, K, mc, cc, c0, pc, mix, q, &Aq, &A0, &Cq, &C0);
    if (mode == 1) {
      const double w = wgt ? wgt[c] : 1.0;
      gA = w * SCq / (SA0 * SC0);
      gC = SAq / (SA0 * SC0);
      if (!cc) gC = 0.0;
    } else {
      if (!(A0 > 0.0) || !(C0 > 0.0)) continue;
      const double norm = A0 * C0;
      *loss += Aq * Cq / norm / (double)n;
      gA = Cq / ((double)n * norm);
      gC = cc ? Aq / ((double)n * norm) : 0.0;
    }
    sample_backward(theta, K, &A, mc, cc, pc, mix, q, gA, gC, dz, gq, grad);
  }
done:
  act_free(&A);
  free(dz);
  free(gq);
  free(q);
  return 0;
}

/* Adam (Kingma & Ba 2015, Algorithm 1), step t >= 1. */
void orc_adam(double *theta, const double *grad, double *m1, double *m2, int64_t n, double lr,
              double beta1, double beta2, double eps, int t) {
  const double c1 = 1.0 - pow(beta1, t), c2 = 1.0 - pow(beta2, t);
  for (int64_t i = 0; i < n; ++i) {
    m1[i] = beta1 * m1[i] + (1.0 - beta1) * grad[i];
    m2[i] = beta2 * m2[i] + (1.0 - beta2) * grad[i] * grad[i];
    const double mh = m1[i] / c1, vh = m2[i] / c2;
    theta[i] -= lr * mh / (sqrt(vh) + eps);
  }
}

/* ---- per-cell integer proposal from probabilities ---------------------------
 * q [n_b n_g] (spectral points, band-major), q_up the upward-hemisphere
 * probability.  The counts of a per-cell proposal are decided in binary32: each
 * probability is rounded to binary32; a band's weight is the binary32 sum of
 * its points in order of g; bands and the g points inside each band are
 * quantised to counts of 2^32 by quantize_f32 (count = floor(RN32(w / W) 2^32)
 * with W the binary32 sum of the weights in order; a point with positive weight
 * keeps at least one count; the rounding remainder goes to the first largest
 * weight); a band whose g weights are all zero gets uniform g counts (it is
 * never drawn).  The hemisphere count of 2^23 is q_up 2^23 rounded half up in
 * binary64, kept in [1, 2^23 - 1].  The plain proposal (orc_plain_proposal)
 * keeps the binary64 rule of orc_quantize. */
static int64_t count_f32(float w, float W) {
  const float y = (w / W) * 4294967296.0f; /* correctly rounded quotient, exact scaling */
  if (y >= 4294967296.0f) return 4294967296LL;
  return (int64_t)(uint32_t)y;             /* y >= 0: truncation is the floor */
}

static int quantize_f32(const float *w, int K, uint64_t *cum) {
  float W = 0.f;
  for (int k = 0; k < K; ++k) W += w[k];
  if (!(W > 0.f)) return -1;
  int kmax = 0;
  for (int k = 1; k < K; ++k)
    if (w[k] > w[kmax]) kmax = k;
  int64_t total = 0;
  for (int k = 0; k < K; ++k) {
    int64_t m = 0;
    if (w[k] > 0.f) {
      m = count_f32(w[k], W);
      if (m < 1) m = 1;
    }
    cum[k] = (uint64_t)m;
    total += m;
  }
  cum[kmax] += (uint64_t)(4294967296LL - total);
  uint64_t acc = 0;
  for (int k = 0; k < K; ++k) {
    acc += cum[k];
    cum[k] = acc;
  }
  return 0;
}

int orc_learned_counts(const double *q, int nb, int ng, double q_up, uint64_t *cn, uint64_t *cg,
                       uint32_t *hemi) {
  float *wn = (float *)malloc(sizeof(float) * nb);
  float *qf = (float *)malloc(sizeof(float) * (size_t)nb * ng);
  float *u = (float *)malloc(sizeof(float) * ng);
  if (!wn || !qf || !u) {
    free(wn);
    free(qf);
    free(u);
    return -1;
  }
  for (size_t i = 0; i < (size_t)nb * ng; ++i) qf[i] = (float)q[i];
  int rc = 0;
  for (int n = 0; n < nb && rc == 0; ++n) {
    float s = 0.f;
    for (int g = 0; g < ng; ++g) s += qf[(size_t)n * ng + g];
    wn[n] = s;
    if (quantize_f32(qf + (size_t)n * ng, ng, cg + (size_t)n * ng) != 0) {
      for (int g = 0; g < ng; ++g) u[g] = 1.f;
      rc = quantize_f32(u, ng, cg + (size_t)n * ng);
    }
  }
  if (rc == 0) rc = quantize_f32(wn, nb, cn);
  double hq = floor(q_up * 8388608.0 + 0.5);
  if (!(hq >= 1.0)) hq = 1.0;
  if (hq > 8388607.0) hq = 8388607.0;
  *hemi = (uint32_t)hq;
  free(wn);
  free(qf);
  free(u);
  return rc;
}

/* ---- spectral proposals at each cell's own temperature ---------------------
 * The classic ERMC draw (Section 2; the paper replaces it by Zhang's T_max pdf,
 * Eq. 13): per cell p(n,g) ~ w_g B_n(T_i) kappa_(n,g)(T_i) (mode 0), or the
 * temperature-weighted mix (1 - lam) p0 + lam p_local with
 * lam = (T_i - T_min) / (T_max - T_min) clamped to [0, 1] (mode 1).  q_out:
 * [n][K] probabilities in FP64. */
int orc_spectral_proposal(const orc_problem *P, int mode, double T_min, double T_max,
                          const double *p0, const int32_t *cells, int64_t n, double *q_out) {
  const int nb = P->n_bands, ng = P->n_g, K = nb * ng;
  for (int64_t q = 0; q < n; ++q) {
    const double T = P->T[cells[q]];
    double *qc = q_out + q * K, W = 0.0;
    for (int b = 0; b < nb; ++b) {
      const double B = orc_interp(P->B + (size_t)b * P->nT, P->T0, P->dT, P->nT, T);
      for (int g = 0; g < ng; ++g) {
        const double k = orc_interp(P->kappa + ((size_t)b * ng + g) * P->nT, P->T0, P->dT, P->nT, T);
        const double v = P->w_g[g] * B * k;
        qc[b * ng + g] = v > 0.0 ? v : 0.0;
        W += qc[b * ng + g];
      }
    }
    double lam = 1.0;
    if (mode == 1) {
      lam = T_max > T_min ? (T - T_min) / (T_max - T_min) : 1.0;
      lam = lam < 0.0 ? 0.0 : (lam > 1.0 ? 1.0 : lam);
    }
    if (!(W > 0.0)) lam = 0.0;
    for (int k = 0; k < K; ++k) qc[k] = (1.0 - lam) * p0[k] + (W > 0.0 ? lam * qc[k] / W : 0.0);
  }
  return 0;
}

