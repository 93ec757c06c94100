// C ABI of the reciprocal Monte Carlo Q_rad library (declared in include/mcrt.h).
//
// Host side only: argument validation, library-owned device buffers, the
// FP64 construction of the quantised spectral proposal (Eq. 13 discretised as
// Eq. 16), and the launches.  Every step of the solve runs in the CUDA kernels
// of trace.cu and fields.cu; nothing here computes Q on the CPU.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "../../include/mcrt.h"
#include "ctx.h"
#include "mcrt_internal.h"
#include "planck.h"

using namespace mcrt_host;

namespace {

bool finite_nonneg(const double *v, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(v[i]) || v[i] < 0.0) return false;
  return true;
}

// Linear interpolation on the uniform T nodes with clamping (Section 2.2).
double interp_host(const double *v, double T0, double dT, int nT, double T) {
  const double f = (T - T0) / dT;
  double t = std::floor(f);
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

// Integer counts of 2^32 proportional to the weights: every positive weight
// gets at least one count (so every contributing (n, g) stays drawable and the
// estimate stays unbiased), the rounding remainder goes to the first largest
// weight.  Writes cumulative counts; false when no weight is positive.
bool quantize_counts(const double *w, int K, unsigned long long *cum) {
  double W = 0.0;
  for (int k = 0; k < K; ++k) W += w[k];
  if (!(W > 0.0)) return false;
  int kmax = 0;
  for (int k = 1; k < K; ++k)
    if (w[k] > w[kmax]) kmax = k;
  std::vector<long long> m(K);
  long long total = 0;
  for (int k = 0; k < K; ++k) {
    if (w[k] > 0.0) {
      const long long mk = (long long)std::floor((w[k] / W) * 4294967296.0);
      m[k] = mk < 1 ? 1 : mk;
    } else {
      m[k] = 0;
    }
    total += m[k];
  }
  m[kmax] += 4294967296LL - total;
  unsigned long long acc = 0;
  for (int k = 0; k < K; ++k) {
    acc += (unsigned long long)m[k];
    cum[k] = acc;
  }
  return true;
}

}  // namespace

namespace mcrt_host {

// Zhang's T_max proposal (Eq. 13) in the narrow-band form of Eq. 16:
// f_n ~ B_n(T_max) sum_g w_g k_{n,g}(T_max) and f_g(n) ~ w_g k_{n,g}(T_max).
int build_plain_proposal(mcrt_ctx *ctx, double Tm, cudaStream_t s) {
  const int nb = ctx->nb, ng = ctx->ng, nT = ctx->nT;
  std::vector<unsigned long long> cn(nb), cg((size_t)nb * ng);
  std::vector<double> wn(nb), wgv(ng);
  for (int n = 0; n < nb; ++n) {
    double sum = 0.0;
    for (int g = 0; g < ng; ++g) {
      wgv[g] = ctx->w_g[g] *
               interp_host(ctx->kappa.data() + ((size_t)n * ng + g) * nT, ctx->T0, ctx->dT, nT, Tm);
      sum += wgv[g];
    }
    wn[n] = interp_host(ctx->B.data() + (size_t)n * nT, ctx->T0, ctx->dT, nT, Tm) * sum;
    if (!quantize_counts(wgv.data(), ng, cg.data() + (size_t)n * ng)) {
      for (int g = 0; g < ng; ++g) wgv[g] = 1.0;  // never drawn; keep rows valid
      quantize_counts(wgv.data(), ng, cg.data() + (size_t)n * ng);
    }
  }
  if (!quantize_counts(wn.data(), nb, cn.data()))
    return fail(ctx, MCRT_E_ARG, "no band emits at T_max (all kappa*B are zero)");
  // ray weights w_g / (p(n,g) q) with q = 1/(4 pi), in FP64, rounded once for the FP32 kernel;
  // the probabilities p(n,g) themselves (FP32) for the learned proposal's mixture
  std::vector<float> w32((size_t)nb * ng);
  ctx->p0_host.assign((size_t)nb * ng, 0.f);
  for (int n = 0; n < nb; ++n)
    for (int g = 0; g < ng; ++g) {
      const unsigned long long mn = cn[n] - (n ? cn[n - 1] : 0ull);
      const unsigned long long mg = cg[(size_t)n * ng + g] - (g ? cg[(size_t)n * ng + g - 1] : 0ull);
      const double p = ((double)mn * 2.3283064365386963e-10) * ((double)mg * 2.3283064365386963e-10);
      w32[(size_t)n * ng + g] = mn && mg ? (float)((ctx->w_g[g] / p) * (6.283185307179586 / 0.5)) : 0.f;
      ctx->p0_host[(size_t)n * ng + g] = (float)p;
    }
  CK(cudaMemcpyAsync(ctx->wgt32.p, w32.data(), sizeof(float) * nb * ng, cudaMemcpyHostToDevice, s),
     "upload weights");
  CK(ensure(ctx->p0_32, sizeof(float) * nb * ng), "alloc plain probabilities");
  CK(cudaMemcpyAsync(ctx->p0_32.p, ctx->p0_host.data(), sizeof(float) * nb * ng, cudaMemcpyHostToDevice, s),
     "upload plain probabilities");
  ctx->p0_T_max = Tm;
  // guide table of the band counts: guide[m] = first band with cum > m 2^32 / G
  const int G = mcrt::fp32_guide_size();
  std::vector<unsigned short> guide(G);
  for (int m = 0, k = 0; m < G; ++m) {
    const unsigned long long lo = (unsigned long long)m << (32 - mcrt::fp32_guide_bits());
    while (cn[k] <= lo) ++k;
    guide[m] = (unsigned short)k;
  }
  CK(cudaMemcpyAsync(ctx->guide.p, guide.data(), sizeof(unsigned short) * G, cudaMemcpyHostToDevice,
                     s),
     "upload guide");
  CK(cudaMemcpyAsync(ctx->cn.p, cn.data(), sizeof(unsigned long long) * nb, cudaMemcpyHostToDevice, s),
     "upload band counts");
  CK(cudaMemcpyAsync(ctx->cg.p, cg.data(), sizeof(unsigned long long) * nb * ng,
                     cudaMemcpyHostToDevice, s),
     "upload g counts");
  // g guides of the bands: gg[n][m] = first g with cum_g(n) > m 2^(32 - bits)
  const int GGn = mcrt::fp32_gguide_size(), ggb = mcrt::fp32_gguide_bits();
  std::vector<unsigned char> gg((size_t)nb * GGn);
  for (int n = 0; n < nb; ++n)
    for (int m = 0, k = 0; m < GGn; ++m) {
      const unsigned long long lo = (unsigned long long)m << (32 - ggb);
      while (cg[(size_t)n * ng + k] <= lo) ++k;
      gg[(size_t)n * GGn + m] = (unsigned char)k;
    }
  CK(cudaMemcpyAsync(ctx->gguide.p, gg.data(), gg.size(), cudaMemcpyHostToDevice, s), "upload g guides");
  // pageable sources: the copies are staged before cudaMemcpyAsync returns
  ctx->prop_valid = true;
  ctx->prop_T_max = Tm;
  return MCRT_OK;
}

}  // namespace mcrt_host

namespace {

// Interpolation positions of the FP32 kernel; valid once both the field and the
// tables are set (recomputed whenever either changes).
int refresh_positions(mcrt_ctx *ctx, cudaStream_t s) {
  if (!ctx->have_kdist || !ctx->have_fields || ctx->nT > 512) return MCRT_OK;
  // every grid of the multigrid march, the problem's own first
  const mcrt_grid_desc &g = ctx->grid;
  const long long n = mcrt::multigrid_cells(g.nx, g.ny, g.nz, mcrt::multigrid_levels(g.nx, g.ny, g.nz));
  CK(ensure(ctx->fpos32, (size_t)n * sizeof(uint2)), "alloc positions");
  CK(mcrt::launch_pack_positions((const double2 *)ctx->field64.p, n, ctx->T0, 1.0 / ctx->dT, ctx->nT,
                                 1.0 / ctx->x_ref, (uint2 *)ctx->fpos32.p, s),
     "pack positions");
  CK(cudaStreamSynchronize(s), "sync");
  return MCRT_OK;
}

}  // namespace

namespace mcrt_host {

double proposal_T_max(const mcrt_ctx *ctx) {
  double Tm = ctx->T_max_field;
  for (int w = 0; w < 2; ++w)
    if (ctx->grid.eps_wall[w] > 0.0 && ctx->grid.T_wall[w] > Tm) Tm = ctx->grid.T_wall[w];
  if (ctx->grid.xz_walls)
    for (int f = 0; f < 4; ++f)
      if (ctx->grid.T_xz[f] > Tm) Tm = ctx->grid.T_xz[f];
  return Tm;
}

int ensure_plain_proposal(mcrt_ctx *ctx, cudaStream_t s) {
  const double Tm = proposal_T_max(ctx);
  if (!ctx->prop_valid || ctx->prop_T_max != Tm || ctx->p0_T_max != Tm)
    return build_plain_proposal(ctx, Tm, s);
  return MCRT_OK;
}

int setup_long_rays(mcrt_ctx *ctx, long long chunk_rays, mcrt::TraceArgs *a) {
  a->long_rays = nullptr;
  a->long_cap = 0;
  a->long_steps = 0x7fffffff;
  a->long_flight = ctx->long_flight;
  if (ctx->long_steps <= 0 || a->mg_levels > 1 || a->xz_walls) return MCRT_OK;
  const long long cap = mcrt::long_ray_capacity(chunk_rays, ctx->long_steps);
  CK(ensure(ctx->longbuf, (size_t)cap * sizeof(mcrt::LongRay)), "alloc long-ray buffer");
  a->long_rays = (mcrt::LongRay *)ctx->longbuf.p;
  a->long_cap = (int)cap;
  a->long_steps = ctx->long_steps;
  return MCRT_OK;
}

int check_solve_params(mcrt_ctx *ctx, const mcrt_solve_params *p, int b[6]) {
  if (p->rays_per_cell < 1) return fail(ctx, MCRT_E_ARG, "rays_per_cell < 1");
  if (p->max_steps < 1) return fail(ctx, MCRT_E_ARG, "max_steps < 1");
  if (!(p->tol > 0.0 && p->tol < 1.0)) return fail(ctx, MCRT_E_ARG, "tol outside (0, 1)");
  if (p->precision != MCRT_FP32 && p->precision != MCRT_FP64)
    return fail(ctx, MCRT_E_ARG, "bad precision");
  if (p->origin != MCRT_ORIGIN_UNIFORM && p->origin != MCRT_ORIGIN_CENTER)
    return fail(ctx, MCRT_E_ARG, "bad origin");
  if (p->proposal != MCRT_PROPOSAL_PLANCK_TMAX && p->proposal != MCRT_PROPOSAL_CELL)
    return fail(ctx, MCRT_E_ARG, "bad proposal");
  if ((unsigned long long)p->ray_offset + (unsigned long long)p->rays_per_cell > (1ull << 32))
    return fail(ctx, MCRT_E_ARG, "ray indices beyond 2^32");
  const mcrt_grid_desc &g = ctx->grid;
  b[0] = 0;
  b[1] = g.nx;
  b[2] = 0;
  b[3] = g.ny;
  b[4] = 0;
  b[5] = g.nz;
  if (p->use_box) {
    std::memcpy(b, p->box, sizeof(int) * 6);
    if (b[0] < 0 || b[1] > g.nx || b[0] > b[1] || b[2] < 0 || b[3] > g.ny || b[2] > b[3] ||
        b[4] < 0 || b[5] > g.nz || b[4] > b[5])
      return fail(ctx, MCRT_E_ARG, "box outside the grid");
  }
  if (!ctx->have_kdist || !ctx->have_fields) return fail(ctx, MCRT_E_STATE, "set kdist and fields first");
  if (p->proposal == MCRT_PROPOSAL_CELL && !ctx->have_cell_prop)
    return fail(ctx, MCRT_E_STATE, "no cell proposal");
  if (p->precision == MCRT_FP32 && ctx->nT > 512)
    return fail(ctx, MCRT_E_UNSUPPORTED, "the FP32 kernel supports tables of at most 512 T nodes");
  if (p->mg_levels < 0 || p->mg_levels > mcrt::multigrid_levels(g.nx, g.ny, g.nz))
    return fail(ctx, MCRT_E_ARG, "mg_levels outside [0, mcrt_multigrid_levels(grid)]");
  if (p->mg_levels > 1 && p->mg_steps < 1) return fail(ctx, MCRT_E_ARG, "mg_steps < 1");
  if (p->estimator != MCRT_EST_ERMC && p->estimator != MCRT_EST_ARMC && p->estimator != MCRT_EST_HYBRID)
    return fail(ctx, MCRT_E_ARG, "bad estimator");
  if (p->estimator != MCRT_EST_ERMC) {
    if (b[0] != 0 || b[1] != g.nx || b[2] != 0 || b[3] != g.ny || b[4] != 0 || b[5] != g.nz)
      return fail(ctx, MCRT_E_UNSUPPORTED, "ARMC / hybrid: the whole grid only (every cell emits)");
    if (p->mg_levels > 1) return fail(ctx, MCRT_E_UNSUPPORTED, "ARMC / hybrid: one grid only");
  }
  return MCRT_OK;
}

// The FP32 kernels' binary32 copies of tol, the cell sizes and the wall
// emissivities (rounded once here).
// The ten Philox4x32-10 round keys of (key0, key1): the Weyl sequence of the
// key schedule (Salmon et al., SC'11) with increments 0x9E3779B9, 0xBB67AE85.
static void set_round_keys(mcrt::TraceArgs *a) {
  unsigned k0 = a->key0, k1 = a->key1;
  for (int r = 0; r < 10; ++r) {
    a->rkey[2 * r] = k0;
    a->rkey[2 * r + 1] = k1;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

static void set_float_copies(mcrt::TraceArgs *a) {
  a->tol32 = (float)a->tol;
  a->dx32 = (float)a->dx;
  a->dy32 = (float)a->dy;
  a->dz32 = (float)a->dz;
  a->eps32[0] = (float)a->eps_wall[0];
  a->eps32[1] = (float)a->eps_wall[1];
}

void fill_trace_args(const mcrt_ctx *ctx, const mcrt_solve_params *p, const int b[6],
                     mcrt::TraceArgs *ap) {
  const mcrt_grid_desc &g = ctx->grid;
  mcrt::TraceArgs &a = *ap;
  std::memset(&a, 0, sizeof(a));
  a.nx = g.nx;
  a.ny = g.ny;
  a.nz = g.nz;
  a.dx = g.lx / g.nx;
  a.dy = g.ly / g.ny;
  a.dz = g.lz / g.nz;
  a.nb = ctx->nb;
  a.ng = ctx->ng;
  a.nT = ctx->nT;
  a.T0 = ctx->T0;
  a.inv_dT = 1.0 / ctx->dT;
  a.inv_xref = 1.0 / ctx->x_ref;
  a.eps_wall[0] = g.eps_wall[0];
  a.eps_wall[1] = g.eps_wall[1];
  a.reflect = g.reflect;
  a.yf64 = (const double *)ctx->yf64.p;
  a.yf32 = (const float *)ctx->yf32.p;
  a.xz_walls = g.xz_walls;
  a.fpos32 = (const uint2 *)ctx->fpos32.p;
  a.field64 = (const double2 *)ctx->field64.p;
  a.ktab32 = (const float2 *)ctx->ktab32.p;
  a.ktab64 = (const double2 *)ctx->ktab64.p;
  a.btab32 = (const float2 *)ctx->btab32.p;
  a.kbtab32 = (const float4 *)ctx->kbtab32.p;
  a.btab64 = (const double2 *)ctx->btab64.p;
  a.bwall32 = (const float *)ctx->bwall32.p;
  a.bwall64 = (const double *)ctx->bwall64.p;
  a.w_g = (const double *)ctx->wg.p;
  a.wgt32 = (const float *)ctx->wgt32.p;
  a.w_g32 = (const float *)ctx->wg32.p;
  a.counts_in_smem = mcrt::fp32_plain_stage_fits(ctx->nb, ctx->ng) ? 1 : 0;
  a.guide = (const unsigned short *)ctx->guide.p;
  a.gguide = (const unsigned char *)ctx->gguide.p;
  a.cn = (const unsigned long long *)ctx->cn.p;
  a.cg = (const unsigned long long *)ctx->cg.p;
  if (p->proposal == MCRT_PROPOSAL_CELL) {
    a.cell_cn = (const unsigned long long *)ctx->cell_cn.p;
    a.cell_cg = (const unsigned long long *)ctx->cell_cg.p;
    a.cell_hemi = (const unsigned int *)ctx->cell_hemi.p;
    if (mcrt::fp32_cell_stage_fits(ctx->nb, ctx->ng)) a.counts_in_smem |= 2;
  }
  a.rays = p->rays_per_cell;
  a.max_steps = p->max_steps;
  a.mg_levels = p->mg_levels > 1 ? p->mg_levels : 1;
  a.mg_steps = p->mg_levels > 1 ? p->mg_steps : 0x7fffffff;
  a.origin = p->origin;
  a.tol = p->tol;
  set_float_copies(&a);
  a.key0 = (unsigned)(p->seed & 0xffffffffu);
  a.key1 = (unsigned)(p->seed >> 32);
  set_round_keys(&a);
  a.claim_rays = ctx->claim_rays;
  a.snapshot = p->snapshot;
  a.ray_offset = p->ray_offset;
  a.bi0 = b[0];
  a.bj0 = b[2];
  a.bk0 = b[4];
  a.bnx = b[1] - b[0];
  a.bny = b[3] - b[2];
  a.bnz = b[5] - b[4];
  a.ncells_box = (long long)a.bnx * a.bny * a.bnz;
  a.counters = (unsigned long long *)ctx->counters.p;
  a.tally32 = ctx->tally32;
  a.reduce_plain = ctx->tally_plain;
}

}  // namespace mcrt_host

extern "C" {

const char *mcrt_status_string(int status) {
  switch (status) {
    case MCRT_OK: return "ok";
    case MCRT_E_ARG: return "invalid argument";
    case MCRT_E_STATE: return "call out of order";
    case MCRT_E_CUDA: return "CUDA error";
    case MCRT_E_OOM: return "device out of memory";
    case MCRT_E_RANGE: return "field value out of range";
    case MCRT_E_TIMEOUT: return "device wait timed out";
    case MCRT_E_UNSUPPORTED: return "unsupported";
    default: return "unknown status";
  }
}

const char *mcrt_last_error(const mcrt_ctx *ctx) { return ctx ? ctx->err.c_str() : ""; }

int mcrt_multigrid_levels(int nx, int ny, int nz) { return mcrt::multigrid_levels(nx, ny, nz); }

int mcrt_create(const mcrt_grid_desc *g, mcrt_ctx **out) {
  if (!out) return MCRT_E_ARG;
  *out = nullptr;
  if (!g) return MCRT_E_ARG;
  if (g->nx < 1 || g->ny < 1 || g->nz < 1) return MCRT_E_ARG;
  if ((long long)g->nx * g->ny * g->nz >= (1LL << 31)) return MCRT_E_ARG;
  if (!(g->lx > 0) || !(g->ly > 0) || !(g->lz > 0) || !std::isfinite(g->lx) ||
      !std::isfinite(g->ly) || !std::isfinite(g->lz))
    return MCRT_E_ARG;
  for (int w = 0; w < 2; ++w) {
    if (!(g->eps_wall[w] >= 0.0 && g->eps_wall[w] <= 1.0)) return MCRT_E_ARG;
    if (!(g->T_wall[w] >= 0.0) || !std::isfinite(g->T_wall[w])) return MCRT_E_ARG;
  }
  if (g->reflect != MCRT_REFLECT_DIFFUSE && g->reflect != MCRT_REFLECT_SPECULAR) return MCRT_E_ARG;
  if (g->xz_walls != 0 && g->xz_walls != 1) return MCRT_E_ARG;
  if (g->xz_walls)
    for (int f = 0; f < 4; ++f)
      if (!(g->T_xz[f] >= 0.0) || !std::isfinite(g->T_xz[f])) return MCRT_E_ARG;
  if (g->yf) {
    // stretched y: 0 = yf[0] < yf[1] < ... < yf[ny] = ly
    if (g->yf[0] != 0.0 || !(std::fabs(g->yf[g->ny] - g->ly) <= 1e-12 * g->ly)) return MCRT_E_ARG;
    for (int j = 0; j < g->ny; ++j)
      if (!(g->yf[j + 1] > g->yf[j]) || !std::isfinite(g->yf[j + 1])) return MCRT_E_ARG;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || g->device < 0 || g->device >= ndev) {
    cudaGetLastError();
    return MCRT_E_CUDA;
  }
  mcrt_ctx *ctx = new (std::nothrow) mcrt_ctx();
  if (!ctx) return MCRT_E_OOM;
  ctx->grid = *g;
  ctx->grid.yf = nullptr;  // the caller's array is not kept
  if (g->yf) {
    ctx->yf.assign(g->yf, g->yf + g->ny + 1);
    ctx->yf.back() = g->ly;
  }
  DeviceGuard dg(g->device);
  if (!dg.ok || cudaEventCreate(&ctx->ev0) != cudaSuccess ||
      cudaEventCreate(&ctx->ev1) != cudaSuccess ||
      ensure(ctx->counters, mcrt::NCOUNTERS * sizeof(unsigned long long)) != cudaSuccess ||
      ensure(ctx->fstats, 3 * sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    mcrt_destroy(ctx);
    return MCRT_E_CUDA;
  }
  if (!ctx->yf.empty()) {
    const size_t nf = ctx->yf.size();
    std::vector<float> f32(ctx->yf.begin(), ctx->yf.end());
    if (ensure(ctx->yf64, nf * sizeof(double)) != cudaSuccess ||
        ensure(ctx->yf32, nf * sizeof(float)) != cudaSuccess ||
        cudaMemcpy(ctx->yf64.p, ctx->yf.data(), nf * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(ctx->yf32.p, f32.data(), nf * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      mcrt_destroy(ctx);
      return MCRT_E_CUDA;
    }
  }
  *out = ctx;
  return MCRT_OK;
}

int mcrt_set_kdist(mcrt_ctx *ctx, const mcrt_kdist_desc *kd_in) {
  if (!ctx) return MCRT_E_ARG;
  if (!kd_in || !kd_in->w_g || !kd_in->kappa) return fail(ctx, MCRT_E_ARG, "null table");
  mcrt_kdist_desc kdv = *kd_in;
  const mcrt_kdist_desc *kd = &kdv;
  if (kd->n_bands < 1 || kd->n_bands > 1024 || kd->n_g < 1 || kd->n_g > 64 || kd->nT < 2 ||
      kd->nT > (1 << 20))
    return fail(ctx, MCRT_E_ARG, "table sizes out of range");
  if (!(kd->dT > 0) || !std::isfinite(kd->dT) || !std::isfinite(kd->T0) || !(kd->x_ref > 0) ||
      !std::isfinite(kd->x_ref))
    return fail(ctx, MCRT_E_ARG, "bad T axis or x_ref");
  std::vector<double> Bcomp;
  if (!kd->B) {
    // the band intensities from the band centres and widths
    if (!kd->nu_c || !kd->dnu) return fail(ctx, MCRT_E_ARG, "B, nu_c or dnu must be given");
    for (int n = 0; n < kd->n_bands; ++n)
      if (!(kd->nu_c[n] > 0.0) || !(kd->dnu[n] > 0.0) || !std::isfinite(kd->nu_c[n]) ||
          !std::isfinite(kd->dnu[n]))
        return fail(ctx, MCRT_E_ARG, "band centres and widths must be positive and finite");
    Bcomp.resize((size_t)kd->n_bands * kd->nT);
    for (int n = 0; n < kd->n_bands; ++n)
      for (int t = 0; t < kd->nT; ++t)
        Bcomp[(size_t)n * kd->nT + t] = mcrt::planck_band(kd->nu_c[n], kd->dnu[n], kd->T0 + t * kd->dT);
    kdv.B = Bcomp.data();
  }
  const int nb = kd->n_bands, ng = kd->n_g, nT = kd->nT;
  const size_t nk = (size_t)nb * ng * nT, nbT = (size_t)nb * nT;
  if (!finite_nonneg(kd->w_g, ng) || !finite_nonneg(kd->kappa, nk) || !finite_nonneg(kd->B, nbT))
    return fail(ctx, MCRT_E_ARG, "negative or non-finite table entry");
  DeviceGuard dg(ctx->grid.device);
  if (!dg.ok) return fail(ctx, MCRT_E_CUDA, "cudaSetDevice");
  ctx->have_kdist = false;
  ctx->prop_valid = false;
  ctx->have_cell_prop = false;
  ctx->nb = nb;
  ctx->ng = ng;
  ctx->nT = nT;
  ctx->T0 = kd->T0;
  ctx->dT = kd->dT;
  ctx->x_ref = kd->x_ref;
  ctx->w_g.assign(kd->w_g, kd->w_g + ng);
  ctx->kappa.assign(kd->kappa, kd->kappa + nk);
  ctx->B.assign(kd->B, kd->B + nbT);
  // interpolation nodes {v_t, v_{t+1} - v_t}; the last node repeats with zero slope
  std::vector<double2> k64(nk), b64(nbT);
  std::vector<float2> k32(nk), b32(nbT);
  for (size_t r = 0; r < (size_t)nb * ng; ++r)
    for (int t = 0; t < nT; ++t) {
      const double v = kd->kappa[r * nT + t];
      const double dv = t + 1 < nT ? kd->kappa[r * nT + t + 1] - v : 0.0;
      k64[r * nT + t] = make_double2(v, dv);
      k32[r * nT + t] = make_float2((float)v, (float)dv);
    }
  for (size_t r = 0; r < (size_t)nb; ++r)
    for (int t = 0; t < nT; ++t) {
      const double v = kd->B[r * nT + t];
      const double dv = t + 1 < nT ? kd->B[r * nT + t + 1] - v : 0.0;
      b64[r * nT + t] = make_double2(v, dv);
      b32[r * nT + t] = make_float2((float)v, (float)dv);
    }
  // band intensity of the six faces: the y walls, then (closed boxes) x and z
  std::vector<double> bw64(6 * (size_t)nb);
  std::vector<float> bw32(6 * (size_t)nb);
  for (int w = 0; w < 6; ++w)
    for (int n = 0; n < nb; ++n) {
      const double Tw = w < 2 ? ctx->grid.T_wall[w] : ctx->grid.T_xz[w - 2];
      bw64[w * nb + n] = interp_host(kd->B + (size_t)n * nT, kd->T0, kd->dT, nT, Tw);
      bw32[w * nb + n] = (float)bw64[w * nb + n];
    }
  CK(ensure(ctx->ktab64, nk * sizeof(double2)), "alloc kappa table");
  CK(ensure(ctx->ktab32, nk * sizeof(float2)), "alloc kappa table");
  CK(ensure(ctx->btab64, nbT * sizeof(double2)), "alloc B table");
  CK(ensure(ctx->btab32, nbT * sizeof(float2)), "alloc B table");
  CK(ensure(ctx->kbtab32, nk * sizeof(float4)), "alloc kappa-B table");
  CK(ensure(ctx->bwall64, 6 * nb * sizeof(double)), "alloc wall B");
  CK(ensure(ctx->bwall32, 6 * nb * sizeof(float)), "alloc wall B");
  CK(ensure(ctx->wg, ng * sizeof(double)), "alloc w_g");
  CK(ensure(ctx->cn, nb * sizeof(unsigned long long)), "alloc band counts");
  CK(ensure(ctx->cg, (size_t)nb * ng * sizeof(unsigned long long)), "alloc g counts");
  CK(ensure(ctx->wgt32, (size_t)nb * ng * sizeof(float)), "alloc weights");
  CK(ensure(ctx->guide, (size_t)mcrt::fp32_guide_size() * sizeof(unsigned short)), "alloc guide");
  CK(ensure(ctx->gguide, (size_t)nb * mcrt::fp32_gguide_size()), "alloc g guides");
  CK(cudaMemcpy(ctx->ktab64.p, k64.data(), nk * sizeof(double2), cudaMemcpyHostToDevice), "copy");
  CK(cudaMemcpy(ctx->ktab32.p, k32.data(), nk * sizeof(float2), cudaMemcpyHostToDevice), "copy");
  CK(cudaMemcpy(ctx->btab64.p, b64.data(), nbT * sizeof(double2), cudaMemcpyHostToDevice), "copy");
  CK(cudaMemcpy(ctx->btab32.p, b32.data(), nbT * sizeof(float2), cudaMemcpyHostToDevice), "copy");
  {
    // the FP32 march's interleaved rows: row (n, g) carries band n's B nodes
    std::vector<float4> kb(nk);
    for (size_t r = 0; r < (size_t)nb * ng; ++r)
      for (int t = 0; t < nT; ++t) {
        const float2 kv = k32[r * nT + t], bv = b32[(r / ng) * nT + t];
        kb[r * nT + t] = make_float4(kv.x, kv.y, bv.x, bv.y);
      }
    CK(cudaMemcpy(ctx->kbtab32.p, kb.data(), nk * sizeof(float4), cudaMemcpyHostToDevice), "copy");
  }
  CK(cudaMemcpy(ctx->bwall64.p, bw64.data(), 6 * nb * sizeof(double), cudaMemcpyHostToDevice), "copy");
  CK(cudaMemcpy(ctx->bwall32.p, bw32.data(), 6 * nb * sizeof(float), cudaMemcpyHostToDevice), "copy");
  CK(cudaMemcpy(ctx->wg.p, kd->w_g, ng * sizeof(double), cudaMemcpyHostToDevice), "copy");
  // Planck-mean coefficients per node (features of the learned proposal)
  std::vector<float4> kp(2 * (size_t)nT);
  for (int t = 0; t < nT; ++t) {
    double N0 = 0, N1 = 0, N2 = 0, D0 = 0, D1 = 0;
    for (int n = 0; n < nb; ++n) {
      const double2 b = b64[(size_t)n * nT + t];
      double S = 0, dS = 0;
      for (int g = 0; g < ng; ++g) {
        const double2 k = k64[((size_t)n * ng + g) * nT + t];
        S += kd->w_g[g] * k.x;
        dS += kd->w_g[g] * k.y;
      }
      N0 += b.x * S;
      N1 += b.x * dS + b.y * S;
      N2 += b.y * dS;
      D0 += b.x;
      D1 += b.y;
    }
    kp[2 * t] = make_float4((float)N0, (float)N1, (float)N2, (float)D0);
    kp[2 * t + 1] = make_float4((float)D1, 0.f, 0.f, 0.f);
  }
  CK(ensure(ctx->kptab, kp.size() * sizeof(float4)), "alloc Planck-mean table");
  CK(cudaMemcpy(ctx->kptab.p, kp.data(), kp.size() * sizeof(float4), cudaMemcpyHostToDevice), "copy");
  std::vector<float> wg32(kd->w_g, kd->w_g + ng);
  CK(ensure(ctx->wg32, ng * sizeof(float)), "alloc w_g");
  CK(cudaMemcpy(ctx->wg32.p, wg32.data(), ng * sizeof(float), cudaMemcpyHostToDevice), "copy");
  ctx->have_kdist = true;
  return refresh_positions(ctx, nullptr);
}

int mcrt_set_fields(mcrt_ctx *ctx, const void *T, const void *x, int fp64, int mem, void *stream) {
  if (!ctx) return MCRT_E_ARG;
  if (!T) return fail(ctx, MCRT_E_ARG, "null T");
  if (mem != MCRT_MEM_HOST && mem != MCRT_MEM_DEVICE) return fail(ctx, MCRT_E_ARG, "bad mem");
  if (fp64 != 0 && fp64 != 1) return fail(ctx, MCRT_E_ARG, "bad dtype flag");
  DeviceGuard dg(ctx->grid.device);
  if (!dg.ok) return fail(ctx, MCRT_E_CUDA, "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  const long long n = (long long)ctx->grid.nx * ctx->grid.ny * ctx->grid.nz;
  const size_t esz = fp64 ? sizeof(double) : sizeof(float);
  ctx->have_fields = false;
  // (the plain proposal depends on the field only through T_max: the solves
  // rebuild it when that changes)
  // field64 also holds the coarser grids of the multigrid march after the
  // problem's own (Section 4.3)
  const int mg_levels = mcrt::multigrid_levels(ctx->grid.nx, ctx->grid.ny, ctx->grid.nz);
  const long long n_all = mcrt::multigrid_cells(ctx->grid.nx, ctx->grid.ny, ctx->grid.nz, mg_levels);
  CK(ensure(ctx->field64, (size_t)n_all * sizeof(double2)), "alloc field");
  const void *dT = T, *dx = x;
  DevBuf &stage = ctx->fstage;  // kept for the next call (no allocation per field update)
  if (mem == MCRT_MEM_HOST) {
    CK(ensure(stage, (size_t)n * esz * (x ? 2 : 1)), "alloc staging");
    CK(cudaMemcpyAsync(stage.p, T, (size_t)n * esz, cudaMemcpyHostToDevice, s), "copy T");
    dT = stage.p;
    if (x) {
      CK(cudaMemcpyAsync((char *)stage.p + (size_t)n * esz, x, (size_t)n * esz,
                         cudaMemcpyHostToDevice, s),
         "copy x");
      dx = (char *)stage.p + (size_t)n * esz;
    }
  }
  if (!x && !ctx->have_kdist) return fail(ctx, MCRT_E_STATE, "x = NULL needs set_kdist first (x_ref)");
  const double x_ref = ctx->have_kdist ? ctx->x_ref : 1.0;
  cudaError_t e = mcrt::launch_pack_fields(dT, dx, fp64, x_ref, n, (double2 *)ctx->field64.p,
                                           (unsigned long long *)ctx->fstats.p, s);
  {
    double2 *lev = (double2 *)ctx->field64.p;
    int d[3] = {ctx->grid.nx, ctx->grid.ny, ctx->grid.nz};
    for (int l = 1; l < mg_levels && e == cudaSuccess; ++l) {
      double2 *next = lev + (size_t)d[0] * d[1] * d[2];
      e = mcrt::launch_coarsen(lev, d[0], d[1], d[2], next, (const double *)ctx->yf64.p, l - 1, s);
      for (int a = 0; a < 3; ++a) d[a] /= 2;
      lev = next;
    }
  }
  unsigned long long st[3] = {0, 0, 0};
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(st, ctx->fstats.p, sizeof(st), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "pack fields");
  if (st[2] != 0)
    return fail(ctx, MCRT_E_RANGE,
                std::to_string(st[2]) + " cells with non-finite or non-positive T or bad x");
  double tmax, tmin;
  std::memcpy(&tmax, &st[0], sizeof(double));
  std::memcpy(&tmin, &st[1], sizeof(double));
  ctx->T_max_field = tmax;
  ctx->T_min_field = tmin;
  ctx->have_fields = true;
  return refresh_positions(ctx, s);
}

int mcrt_set_cell_proposal(mcrt_ctx *ctx, const uint64_t *cn, const uint64_t *cg,
                           const uint32_t *hemi, int mem, void *stream) {
  if (!ctx) return MCRT_E_ARG;
  if (!ctx->have_kdist) return fail(ctx, MCRT_E_STATE, "set_kdist first");
  if (!cn || !cg || !hemi) return fail(ctx, MCRT_E_ARG, "null proposal array");
  if (mem != MCRT_MEM_HOST && mem != MCRT_MEM_DEVICE) return fail(ctx, MCRT_E_ARG, "bad mem");
  DeviceGuard dg(ctx->grid.device);
  if (!dg.ok) return fail(ctx, MCRT_E_CUDA, "cudaSetDevice");
  const size_t nc = (size_t)ctx->grid.nx * ctx->grid.ny * ctx->grid.nz;
  const size_t nb = ctx->nb, ng = ctx->ng;
  if (mem == MCRT_MEM_HOST) {
    for (size_t c = 0; c < nc; ++c) {
      const uint64_t *a = cn + c * nb;
      if (a[nb - 1] != (1ull << 32)) return fail(ctx, MCRT_E_ARG, "band counts must end at 2^32");
      for (size_t k = 1; k < nb; ++k)
        if (a[k] < a[k - 1]) return fail(ctx, MCRT_E_ARG, "band counts decrease");
      for (size_t n = 0; n < nb; ++n) {
        const uint64_t *b = cg + (c * nb + n) * ng;
        if (b[ng - 1] != (1ull << 32)) return fail(ctx, MCRT_E_ARG, "g counts must end at 2^32");
        for (size_t k = 1; k < ng; ++k)
          if (b[k] < b[k - 1]) return fail(ctx, MCRT_E_ARG, "g counts decrease");
      }
      if (hemi[c] < 1u || hemi[c] >= (1u << 23))
        return fail(ctx, MCRT_E_ARG, "hemisphere count outside [1, 2^23-1]");
    }
  }
  ctx->have_cell_prop = false;
  cudaStream_t s = (cudaStream_t)stream;
  CK(ensure(ctx->cell_cn, nc * nb * sizeof(uint64_t)), "alloc cell proposal");
  CK(ensure(ctx->cell_cg, nc * nb * ng * sizeof(uint64_t)), "alloc cell proposal");
  CK(ensure(ctx->cell_hemi, nc * sizeof(uint32_t)), "alloc cell proposal");
  const cudaMemcpyKind k = mem == MCRT_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  CK(cudaMemcpyAsync(ctx->cell_cn.p, cn, nc * nb * sizeof(uint64_t), k, s), "copy cn");
  CK(cudaMemcpyAsync(ctx->cell_cg.p, cg, nc * nb * ng * sizeof(uint64_t), k, s), "copy cg");
  CK(cudaMemcpyAsync(ctx->cell_hemi.p, hemi, nc * sizeof(uint32_t), k, s), "copy hemi");
  CK(cudaStreamSynchronize(s), "sync");
  ctx->have_cell_prop = true;
  return MCRT_OK;
}

int mcrt_solve_qrad(mcrt_ctx *ctx, const mcrt_solve_params *p, double *q_out, double *sigma_out,
                    int mem, void *stream) {
  if (!ctx) return MCRT_E_ARG;
  if (!p || !q_out) return fail(ctx, MCRT_E_ARG, "null params or q_out");
  if (mem != MCRT_MEM_HOST && mem != MCRT_MEM_DEVICE) return fail(ctx, MCRT_E_ARG, "bad mem");
  int b[6];
  const int rc0 = check_solve_params(ctx, p, b);
  if (rc0 != MCRT_OK) return rc0;
  DeviceGuard dg(ctx->grid.device);
  if (!dg.ok) return fail(ctx, MCRT_E_CUDA, "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;

  const int rcp = ensure_plain_proposal(ctx, s);
  if (rcp != MCRT_OK) return rcp;
  const double Tm = ctx->prop_T_max;
  const long long nbox = (long long)(b[1] - b[0]) * (b[3] - b[2]) * (b[5] - b[4]);

  mcrt::TraceArgs a;
  fill_trace_args(ctx, p, b, &a);

  double *dq = q_out, *ds = sigma_out;
  unsigned long long *dst = (unsigned long long *)p->steps_out;
  if (mem == MCRT_MEM_HOST && nbox > 0) {
    CK(ensure(ctx->q, nbox * sizeof(double)), "alloc q");
    dq = (double *)ctx->q.p;
    if (sigma_out) {
      CK(ensure(ctx->sigma, nbox * sizeof(double)), "alloc sigma");
      ds = (double *)ctx->sigma.p;
    }
    if (p->steps_out) {
      CK(ensure(ctx->steps, nbox * sizeof(unsigned long long)), "alloc steps");
      dst = (unsigned long long *)ctx->steps.p;
    }
  }
  a.q = dq;
  a.sigma = ds;
  a.steps_cell = dst;

  CK(cudaMemsetAsync(ctx->counters.p, 0, mcrt::NCOUNTERS * sizeof(unsigned long long), s), "clear counters");
  int launches = 0;
  if (p->precision == MCRT_FP32 && nbox > 0) {
    // brick-ordered positions in chunks whose per-ray samples fit the scratch
    const long long P = mcrt::fp32_bricks_positions(a.bnx, a.bny, a.bnz);
    const long long cap = (long long)ctx->scratch_mib << 20;
    long long Pc = cap / ((long long)p->rays_per_cell * (long long)sizeof(float));
    if (Pc < 1) Pc = 1;
    if (Pc > P) Pc = P;
    CK(ensure(ctx->ybuf, (size_t)Pc * p->rays_per_cell * sizeof(float)), "alloc sample scratch");
    CK(ensure(ctx->step_acc, (size_t)Pc * sizeof(unsigned long long)), "alloc step scratch");
    a.ybuf = (float *)ctx->ybuf.p;
    a.step_acc = (unsigned long long *)ctx->step_acc.p;
    // cells of more than one tally segment: each segment summed by a warp of its own
    const int nseg = mcrt::tally_segments((p->rays_per_cell + 31) / 32);
    a.tally_part = nullptr;
    if (nseg > 1 && !ctx->tally32) {
      CK(ensure(ctx->tpart, (size_t)Pc * (size_t)nseg * sizeof(double2)), "alloc tally segments");
      a.tally_part = (double2 *)ctx->tpart.p;
    }
    const int rl = setup_long_rays(ctx, Pc * (long long)p->rays_per_cell, &a);
    if (rl != MCRT_OK) return rl;
    const bool armc = p->estimator != MCRT_EST_ERMC;
    const long long ncg = (long long)ctx->grid.nx * ctx->grid.ny * ctx->grid.nz;
    if (armc) {
      // per-batch sums of the deposits and of the cells' own samples (the
      // long-ray march makes the deposits of the rays handed to it)
      CK(ensure(ctx->armcbuf, (size_t)2 * 16 * ncg * sizeof(double)), "alloc ARMC sums");
      CK(cudaMemsetAsync(ctx->armcbuf.p, 0, (size_t)2 * 16 * ncg * sizeof(double), s), "clear ARMC sums");
      a.armc_acc = (double *)ctx->armcbuf.p;
      a.ermc_acc = a.armc_acc + 16 * ncg;
      a.armc_nc = ncg;
    }
    const int nchunks = (int)((P + Pc - 1) / Pc);
    while ((int)ctx->kev.size() < 4 * nchunks) {
      cudaEvent_t e = nullptr;
      CK(cudaEventCreate(&e), "event");
      ctx->kev.push_back(e);
    }
    ctx->kev_chunks = 0;
    CK(cudaEventRecord(ctx->ev0, s), "event");
    for (long long p0 = 0; p0 < P; p0 += Pc) {
      a.chunk_p0 = p0;
      a.chunk_p1 = p0 + Pc < P ? p0 + Pc : P;
      if (dst)
        CK(cudaMemsetAsync(ctx->step_acc.p, 0, (size_t)(a.chunk_p1 - p0) * sizeof(unsigned long long), s),
           "clear step scratch");
      int kn = 0;
      CK(mcrt::launch_trace_fp32(a, ctx->min_blocks, ctx->steps_per_round, s,
                                 ctx->kev.data() + 4 * ctx->kev_chunks, &kn),
         "trace launch");
      ++ctx->kev_chunks;
      launches += kn;
    }
    if (armc) {
      CK(mcrt::launch_armc_finalize(a.armc_acc, a.ermc_acc, ncg, p->rays_per_cell < 16 ? p->rays_per_cell : 16,
                                    p->rays_per_cell, p->estimator == MCRT_EST_HYBRID,
                                    (const double2 *)ctx->field64.p, ctx->T_min_field, ctx->T_max_field, dq, ds,
                                    s),
         "ARMC finalize");
      ++launches;
    }
    CK(cudaEventRecord(ctx->ev1, s), "event");
  } else {
    const bool armc = p->estimator != MCRT_EST_ERMC && nbox > 0;
    const long long ncg = (long long)ctx->grid.nx * ctx->grid.ny * ctx->grid.nz;
    if (armc) {  // as in the FP32 solve
      CK(ensure(ctx->armcbuf, (size_t)2 * 16 * ncg * sizeof(double)), "alloc ARMC sums");
      CK(cudaMemsetAsync(ctx->armcbuf.p, 0, (size_t)2 * 16 * ncg * sizeof(double), s), "clear ARMC sums");
      a.armc_acc = (double *)ctx->armcbuf.p;
      a.ermc_acc = a.armc_acc + 16 * ncg;
      a.armc_nc = ncg;
    }
    ctx->kev_chunks = 0;
    CK(cudaEventRecord(ctx->ev0, s), "event");
    CK(mcrt::launch_trace(a, p->precision, s), "trace launch");
    launches = nbox > 0 ? 1 : 0;
    if (armc) {
      CK(mcrt::launch_armc_finalize(a.armc_acc, a.ermc_acc, ncg, p->rays_per_cell < 16 ? p->rays_per_cell : 16,
                                    p->rays_per_cell, p->estimator == MCRT_EST_HYBRID,
                                    (const double2 *)ctx->field64.p, ctx->T_min_field, ctx->T_max_field, dq, ds,
                                    s),
         "ARMC finalize");
      ++launches;
    }
    CK(cudaEventRecord(ctx->ev1, s), "event");
  }
  ctx->last_launches = launches;
  ctx->last_stream = s;
  ctx->solved = true;
  ctx->last_T_max = Tm;
  if (mem == MCRT_MEM_HOST && nbox > 0) {
    CK(cudaMemcpyAsync(q_out, dq, nbox * sizeof(double), cudaMemcpyDeviceToHost, s), "copy q");
    if (sigma_out)
      CK(cudaMemcpyAsync(sigma_out, ds, nbox * sizeof(double), cudaMemcpyDeviceToHost, s),
         "copy sigma");
    if (p->steps_out)
      CK(cudaMemcpyAsync(p->steps_out, dst, nbox * sizeof(unsigned long long),
                         cudaMemcpyDeviceToHost, s),
         "copy steps");
    unsigned long long flag = 0;
    CK(cudaMemcpyAsync(&flag, (unsigned long long *)ctx->counters.p + 5, sizeof(flag),
                       cudaMemcpyDeviceToHost, s),
       "read error flag");
    CK(cudaStreamSynchronize(s), "sync");
    if (flag != 0) return fail(ctx, MCRT_E_TIMEOUT, "a device-side wait gave up (trace or tally kernel)");
  }
  return MCRT_OK;
}

int mcrt_set_tuning(mcrt_ctx *ctx, const mcrt_tuning *t) {
  if (!ctx) return MCRT_E_ARG;
  if (!t) return fail(ctx, MCRT_E_ARG, "null tuning");
  if (t->min_blocks_per_sm < 0 || t->min_blocks_per_sm > 4)
    return fail(ctx, MCRT_E_ARG, "min_blocks_per_sm outside 0..4");
  if (t->scratch_mib < 0 || t->scratch_mib > (1 << 20))
    return fail(ctx, MCRT_E_ARG, "scratch_mib outside 0..2^20");
  if (t->steps_per_round != 0 && t->steps_per_round != 1 && t->steps_per_round != 2 &&
      t->steps_per_round != 4)
    return fail(ctx, MCRT_E_ARG, "steps_per_round not in {0, 1, 2, 4}");
  if (t->long_ray_flight > (1 << 24)) return fail(ctx, MCRT_E_ARG, "long_ray_flight above 2^24");
  if (t->tally_binary32 != 0 && t->tally_binary32 != 1) return fail(ctx, MCRT_E_ARG, "tally_binary32 not 0 or 1");
  if (t->tally_plain_loads != 0 && t->tally_plain_loads != 1)
    return fail(ctx, MCRT_E_ARG, "tally_plain_loads not 0 or 1");
  if (t->claim_rays != 0 && (t->claim_rays < 32 || t->claim_rays > (1 << 20)))
    return fail(ctx, MCRT_E_ARG, "claim_rays not 0 or within 32..2^20");
  if (t->batch_per_snapshot != 0 && t->batch_per_snapshot != 1)
    return fail(ctx, MCRT_E_ARG, "batch_per_snapshot not 0 or 1");
  ctx->min_blocks = t->min_blocks_per_sm ? t->min_blocks_per_sm : 3;
  ctx->steps_per_round = t->steps_per_round ? t->steps_per_round : 1;
  ctx->scratch_mib = t->scratch_mib ? t->scratch_mib : 4096;
  ctx->long_steps = t->long_ray_steps ? (t->long_ray_steps > 0 ? t->long_ray_steps : -1) : 1024;
  ctx->long_flight = t->long_ray_flight ? (t->long_ray_flight > 0 ? (float)t->long_ray_flight : -1.f) : 32.f;
  ctx->tally32 = t->tally_binary32;
  ctx->batch_per_snapshot = t->batch_per_snapshot;
  ctx->claim_rays = t->claim_rays ? t->claim_rays : 1024;
  ctx->tally_plain = t->tally_plain_loads;
  return MCRT_OK;
}

int mcrt_get_tuning(const mcrt_ctx *ctx, mcrt_tuning *t) {
  if (!ctx || !t) return MCRT_E_ARG;
  t->min_blocks_per_sm = ctx->min_blocks;
  t->steps_per_round = ctx->steps_per_round;
  t->scratch_mib = ctx->scratch_mib;
  t->long_ray_steps = ctx->long_steps;
  t->long_ray_flight = ctx->long_flight < 0.f ? -1 : (int)ctx->long_flight;
  t->tally_binary32 = ctx->tally32;
  t->batch_per_snapshot = ctx->batch_per_snapshot;
  t->claim_rays = ctx->claim_rays;
  t->tally_plain_loads = ctx->tally_plain;
  return MCRT_OK;
}

int mcrt_get_stats(mcrt_ctx *ctx, mcrt_solve_stats *out) {
  if (!ctx) return MCRT_E_ARG;
  if (!out) return fail(ctx, MCRT_E_ARG, "null out");
  if (!ctx->solved) return fail(ctx, MCRT_E_STATE, "no solve yet");
  DeviceGuard dg(ctx->grid.device);
  if (!dg.ok) return fail(ctx, MCRT_E_CUDA, "cudaSetDevice");
  unsigned long long c[mcrt::NCOUNTERS];
  CK(cudaMemcpyAsync(c, ctx->counters.p, sizeof(c), cudaMemcpyDeviceToHost, ctx->last_stream),
     "read counters");
  CK(cudaStreamSynchronize(ctx->last_stream), "sync");
  if (c[5] != 0) return fail(ctx, MCRT_E_TIMEOUT, "a device-side wait gave up (trace or tally kernel)");
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1), "elapsed");
  out->steps = c[0];
  out->capped = c[1];
  out->wall_hits = c[2];
  out->max_ray_steps = c[4];
  out->rays = c[3];
  out->T_max = ctx->last_T_max;
  out->kernel_ms = ms;
  out->launches = ctx->last_launches;
  out->long_rays = c[8];
  out->long_overflow = c[9];
  out->trace_ms = out->long_ms = out->reduce_ms = 0.f;
  for (int k = 0; k < ctx->kev_chunks; ++k) {
    float t[3];
    for (int j = 0; j < 3; ++j)
      CK(cudaEventElapsedTime(&t[j], ctx->kev[4 * k + j], ctx->kev[4 * k + j + 1]), "elapsed");
    out->trace_ms += t[0];
    out->long_ms += t[1];
    out->reduce_ms += t[2];
  }
  return MCRT_OK;
}

int mcrt_destroy(mcrt_ctx *ctx) {
  if (!ctx) return MCRT_OK;
  {
    DeviceGuard dg(ctx->grid.device);
    cudaDeviceSynchronize();
    DevBuf *bufs[] = {&ctx->yf64, &ctx->yf32, &ctx->longbuf, &ctx->armcbuf, &ctx->fstage, &ctx->tpart, &ctx->field64, &ctx->fpos32, &ctx->ktab64, &ctx->ktab32, &ctx->kbtab32, &ctx->btab64,
                      &ctx->btab32, &ctx->bwall64, &ctx->bwall32, &ctx->wg, &ctx->wg32, &ctx->wgt32, &ctx->cn, &ctx->guide, &ctx->gguide, &ctx->ybuf, &ctx->step_acc,
                      &ctx->cg, &ctx->cell_cn, &ctx->cell_cg, &ctx->cell_hemi,
                      &ctx->counters, &ctx->fstats, &ctx->q, &ctx->sigma, &ctx->steps,
                      &ctx->p0_32, &ctx->feat, &ctx->ray_steps, &ctx->lerr, &ctx->kptab, &ctx->qprop};
    for (DevBuf *b : bufs) release(*b);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    for (cudaEvent_t e : ctx->kev) cudaEventDestroy(e);
    cudaGetLastError();
  }
  delete ctx;
  return MCRT_OK;
}

}  // extern "C"

// ---- allocation-free solve (no counterpart in the paper) ----------------------

namespace {

// Plain-proposal counts, weights and guide table built from fixed host buffers
// (no heap or device allocation) into the context's existing device buffers.
// Same construction as build_plain_proposal.
int noalloc_build_plain_proposal(mcrt_ctx *ctx, double Tm, cudaStream_t s) {
  static std::mutex mu;
  static unsigned long long cn[1024], cg[1024 * 64];
  static double wn[1024], wgv[64], wtmp[64];
  static float w32[1024 * 64];
  static unsigned short guide[4096];  // at least fp32_guide_size() entries
  static unsigned char gg[1024 * 32];  // at least n_bands x fp32_gguide_size()
  std::lock_guard<std::mutex> lock(mu);
  const int nb = ctx->nb, ng = ctx->ng, nT = ctx->nT;
  for (int n = 0; n < nb; ++n) {
    double sum = 0.0;
    for (int g = 0; g < ng; ++g) {
      wgv[g] = ctx->w_g[g] *
               interp_host(ctx->kappa.data() + ((size_t)n * ng + g) * nT, ctx->T0, ctx->dT, nT, Tm);
      sum += wgv[g];
    }
    wn[n] = interp_host(ctx->B.data() + (size_t)n * nT, ctx->T0, ctx->dT, nT, Tm) * sum;
    if (!quantize_counts(wgv, ng, cg + (size_t)n * ng)) {
      for (int g = 0; g < ng; ++g) wtmp[g] = 1.0;  // never drawn; keep rows valid
      quantize_counts(wtmp, ng, cg + (size_t)n * ng);
    }
  }
  if (!quantize_counts(wn, nb, cn))
    return fail(ctx, MCRT_E_ARG, "no band emits at T_max (all kappa*B are zero)");
  for (int n = 0; n < nb; ++n)
    for (int g = 0; g < ng; ++g) {
      const unsigned long long mn = cn[n] - (n ? cn[n - 1] : 0ull);
      const unsigned long long mg = cg[(size_t)n * ng + g] - (g ? cg[(size_t)n * ng + g - 1] : 0ull);
      const double p = ((double)mn * 2.3283064365386963e-10) * ((double)mg * 2.3283064365386963e-10);
      w32[(size_t)n * ng + g] = mn && mg ? (float)((ctx->w_g[g] / p) * (6.283185307179586 / 0.5)) : 0.f;
    }
  const int G = mcrt::fp32_guide_size();
  for (int m = 0, k = 0; m < G; ++m) {
    const unsigned long long lo = (unsigned long long)m << (32 - mcrt::fp32_guide_bits());
    while (cn[k] <= lo) ++k;
    guide[m] = (unsigned short)k;
  }
  // pageable sources: each copy is staged before cudaMemcpyAsync returns
  CK(cudaMemcpyAsync(ctx->wgt32.p, w32, sizeof(float) * nb * ng, cudaMemcpyHostToDevice, s), "weights");
  CK(cudaMemcpyAsync(ctx->guide.p, guide, sizeof(unsigned short) * G, cudaMemcpyHostToDevice, s), "guide");
  CK(cudaMemcpyAsync(ctx->cn.p, cn, sizeof(unsigned long long) * nb, cudaMemcpyHostToDevice, s), "counts");
  CK(cudaMemcpyAsync(ctx->cg.p, cg, sizeof(unsigned long long) * nb * ng, cudaMemcpyHostToDevice, s),
     "counts");
  const int GGn = mcrt::fp32_gguide_size(), ggb = mcrt::fp32_gguide_bits();
  for (int n = 0; n < nb; ++n)
    for (int m = 0, k = 0; m < GGn; ++m) {
      const unsigned long long lo = (unsigned long long)m << (32 - ggb);
      while (cg[(size_t)n * ng + k] <= lo) ++k;
      gg[(size_t)n * GGn + m] = (unsigned char)k;
    }
  CK(cudaMemcpyAsync(ctx->gguide.p, gg, (size_t)nb * GGn, cudaMemcpyHostToDevice, s), "g guides");
  ctx->prop_valid = true;
  ctx->prop_T_max = Tm;
  return MCRT_OK;
}

}  // namespace

extern "C" int mcrt_solve_qrad_noalloc(mcrt_ctx *ctx, const mcrt_solve_params *p, double *q_out,
                                       double *sigma_out, void *stream) {
  if (!ctx) return MCRT_E_ARG;
  if (!p || !q_out) return fail(ctx, MCRT_E_ARG, "null params or q_out");
  if (p->precision != MCRT_FP32) return fail(ctx, MCRT_E_ARG, "the allocation-free solve is FP32 only");
  if (p->estimator != MCRT_EST_ERMC)
    return fail(ctx, MCRT_E_UNSUPPORTED, "the allocation-free solve is emission-based only");
  int b[6];
  const int rc0 = check_solve_params(ctx, p, b);
  if (rc0 != MCRT_OK) return rc0;
  // scratch layout in the static array: counters | long rays | per-position step
  // sums | samples.  The long-ray region holds the smallest buffer a regular
  // solve uses, so both hand the same rays off and give the same bits.
  const size_t total = mcrt::noalloc_scratch_bytes();
  const bool long_on = ctx->long_steps > 0 && p->mg_levels <= 1 && !ctx->grid.xz_walls;
  const long long long_cap = long_on ? 65536 : 0;  // the least capacity of a regular solve's buffer (8 MiB)
  const size_t head_bytes = 256 + (size_t)long_cap * sizeof(mcrt::LongRay);
  const size_t per_pos = (size_t)p->rays_per_cell * sizeof(float) + sizeof(unsigned long long);
  if (total < head_bytes + 256 + per_pos)
    return fail(ctx, MCRT_E_ARG,
                "rays_per_cell too large for the static scratch of the allocation-free solve (" +
                    std::to_string(total >> 20) + " MiB: at most " +
                    std::to_string((total - head_bytes - 256 - sizeof(unsigned long long)) / sizeof(float)) +
                    " rays per cell)");
  DeviceGuard dg(ctx->grid.device);
  if (!dg.ok) return fail(ctx, MCRT_E_CUDA, "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  void *base = nullptr;
  CK(mcrt::noalloc_scratch(ctx->grid.device, &base), "static scratch address");

  const double Tm = proposal_T_max(ctx);
  if (!ctx->prop_valid || ctx->prop_T_max != Tm) {
    const int rc = noalloc_build_plain_proposal(ctx, Tm, s);
    if (rc != MCRT_OK) return rc;
  }
  const long long nbox = (long long)(b[1] - b[0]) * (b[3] - b[2]) * (b[5] - b[4]);
  if (nbox == 0) return MCRT_OK;

  // the regular solve's launch arguments; only the scratch and outputs differ
  mcrt::TraceArgs a;
  fill_trace_args(ctx, p, b, &a);
  a.q = q_out;
  a.sigma = sigma_out;
  a.steps_cell = (unsigned long long *)p->steps_out;

  // carve the static array; positions per chunk as many as fit
  const long long P = mcrt::fp32_bricks_positions(a.bnx, a.bny, a.bnz);
  long long Pc = (long long)((total - head_bytes - 256) / per_pos);
  if (Pc > P) Pc = P;
  unsigned char *cbase = (unsigned char *)base;
  a.counters = (unsigned long long *)cbase;
  a.long_rays = long_on ? (mcrt::LongRay *)(cbase + 256) : nullptr;
  a.long_cap = (int)long_cap;
  a.long_steps = long_on ? ctx->long_steps : 0x7fffffff;
  a.long_flight = ctx->long_flight;
  a.step_acc = (unsigned long long *)(cbase + head_bytes);
  const size_t ybuf_off = (head_bytes + (size_t)Pc * sizeof(unsigned long long) + 255) & ~(size_t)255;
  a.ybuf = (float *)(cbase + ybuf_off);
  CK(cudaMemsetAsync(a.counters, 0, mcrt::NCOUNTERS * sizeof(unsigned long long), s), "clear counters");
  for (long long p0 = 0; p0 < P; p0 += Pc) {
    a.chunk_p0 = p0;
    a.chunk_p1 = p0 + Pc < P ? p0 + Pc : P;
    if (a.steps_cell)
      CK(cudaMemsetAsync(a.step_acc, 0, (size_t)(a.chunk_p1 - p0) * sizeof(unsigned long long), s),
         "clear step sums");
    CK(mcrt::launch_trace_fp32(a, ctx->min_blocks, ctx->steps_per_round, s), "trace launch");
  }
  return MCRT_OK;
}

// ---- batched snapshots in one graph launch ------------------------------------

struct mcrt_batch {
  int device = 0;
  std::vector<mcrt_ctx *> ctxs;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> joins;
  cudaEvent_t fork = nullptr, ev0 = nullptr, ev1 = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  unsigned long long *d_offset = nullptr;
  unsigned long long h_offset = 0;
  std::vector<void *> owned;           // per-branch sample scratch and step sums, per-item counters
  std::vector<unsigned long long *> counters;
  int rays = 0;
  int launches = 0;
  bool single_launch = false;  // one persistent trace launch over every snapshot
  bool ran = false;
  cudaStream_t last_stream = nullptr;
  std::string err;
};

namespace {

int batch_fail(mcrt_batch *b, int code, const std::string &msg) {
  if (b) b->err = msg;
  return code;
}

void batch_release(mcrt_batch *b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (cudaStream_t st : b->streams)
    if (st) cudaStreamDestroy(st);
  for (cudaEvent_t e : b->joins)
    if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  if (b->d_offset) cudaFree(b->d_offset);
  for (void *q : b->owned)
    if (q) cudaFree(q);
  cudaGetLastError();
}

}  // namespace

extern "C" int mcrt_batch_create(const mcrt_batch_item *items, int n, const mcrt_solve_params *p,
                                 const double *weights, int streams, mcrt_batch **out) {
  if (!out) return MCRT_E_ARG;
  *out = nullptr;
  if (!items || n < 1 || !p || streams < 1) return MCRT_E_ARG;
  if (streams > n) streams = n;
  if (p->precision != MCRT_FP32 || p->rays_per_cell < 1 || p->max_steps < 1 ||
      !(p->tol > 0.0 && p->tol < 1.0) || (p->origin != MCRT_ORIGIN_UNIFORM && p->origin != MCRT_ORIGIN_CENTER) ||
      (p->proposal != MCRT_PROPOSAL_PLANCK_TMAX && p->proposal != MCRT_PROPOSAL_CELL) ||
      p->estimator != MCRT_EST_ERMC)
    return MCRT_E_ARG;
  const int dev = items[0].ctx ? items[0].ctx->grid.device : -1;
  for (int k = 0; k < n; ++k) {
    mcrt_ctx *c = items[k].ctx;
    if (!c || !items[k].q_out) return MCRT_E_ARG;
    if (c->grid.device != dev) return fail(c, MCRT_E_ARG, "batch items on different devices");
    if (!c->have_kdist || !c->have_fields) return fail(c, MCRT_E_STATE, "set kdist and fields first");
    if (c->nT > 512) return fail(c, MCRT_E_UNSUPPORTED, "the FP32 kernel supports at most 512 T nodes");
    if (p->proposal == MCRT_PROPOSAL_CELL && !c->have_cell_prop)
      return fail(c, MCRT_E_STATE, "no cell proposal");
    if (weights && !(weights[k] > 0.0) ) return fail(c, MCRT_E_ARG, "batch weights must be > 0");
    if (p->mg_levels < 0 || p->mg_levels > mcrt::multigrid_levels(c->grid.nx, c->grid.ny, c->grid.nz) ||
        (p->mg_levels > 1 && p->mg_steps < 1))
      return fail(c, MCRT_E_ARG, "mg_levels outside [0, mcrt_multigrid_levels(grid)] or mg_steps < 1");
    for (int j = 0; j < k; ++j)
      if (items[j].ctx == c) return fail(c, MCRT_E_ARG, "a context appears twice in the batch");
  }
  mcrt_batch *b = new (std::nothrow) mcrt_batch();
  if (!b) return MCRT_E_OOM;
  b->device = dev;
  b->rays = p->rays_per_cell;
  DeviceGuard dg(dev);
  auto bail = [&](int code, cudaError_t e, const char *where) {
    cudaGetLastError();
    mcrt_ctx *c0 = items[0].ctx;
    fail(c0, code, std::string(where) + (e != cudaSuccess ? std::string(": ") + cudaGetErrorString(e) : ""));
    batch_release(b);
    delete b;
    return code;
  };
#define BK(call, where)                                                                     \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) return bail(e_ == cudaErrorMemoryAllocation ? MCRT_E_OOM : MCRT_E_CUDA, e_, where); \
  } while (0)
  if (!dg.ok) return bail(MCRT_E_CUDA, cudaSuccess, "cudaSetDevice");
  BK(cudaMalloc(&b->d_offset, sizeof(unsigned long long)), "alloc offset");
  BK(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming), "event");
  BK(cudaEventCreate(&b->ev0), "event");
  BK(cudaEventCreate(&b->ev1), "event");
  // per-item preparation: proposal, scratch, launch arguments
  std::vector<mcrt::TraceArgs> args(n);
  std::vector<long long> P(n), Pc(n);
  double wsum = 0.0;
  std::vector<double> w(n);
  for (int k = 0; k < n; ++k) {
    mcrt_ctx *c = items[k].ctx;
    b->ctxs.push_back(c);
    const double Tm = proposal_T_max(c);
    if (!c->prop_valid || c->prop_T_max != Tm) {
      const int rc = build_plain_proposal(c, Tm, nullptr);
      if (rc != MCRT_OK) return bail(rc, cudaSuccess, "proposal");
    }
    const mcrt_grid_desc &g = c->grid;
    mcrt::TraceArgs &a = args[k];
    std::memset(&a, 0, sizeof(a));
    a.tally32 = items[0].ctx->tally32;
    // per-item launches run side by side in graph branches: their tallies take
    // the plain-load kernel, whose blocks (37 KB of shared memory) share the SMs
    // with the other branches' trace kernels more easily than the TMA-fed one's
    // (67 KB): 464 against 479 ms on 8 branches of 32 snapshots
    a.reduce_plain = 1;
    a.nx = g.nx;
    a.ny = g.ny;
    a.nz = g.nz;
    a.dx = g.lx / g.nx;
    a.dy = g.ly / g.ny;
    a.dz = g.lz / g.nz;
    a.nb = c->nb;
    a.ng = c->ng;
    a.nT = c->nT;
    a.T0 = c->T0;
    a.inv_dT = 1.0 / c->dT;
    a.inv_xref = 1.0 / c->x_ref;
    a.eps_wall[0] = g.eps_wall[0];
    a.eps_wall[1] = g.eps_wall[1];
    a.reflect = g.reflect;
    a.yf64 = (const double *)c->yf64.p;
    a.yf32 = (const float *)c->yf32.p;
    a.xz_walls = g.xz_walls;
    a.fpos32 = (const uint2 *)c->fpos32.p;
    a.ktab32 = (const float2 *)c->ktab32.p;
    a.btab32 = (const float2 *)c->btab32.p;
    a.kbtab32 = (const float4 *)c->kbtab32.p;
    a.bwall32 = (const float *)c->bwall32.p;
    a.w_g = (const double *)c->wg.p;
    a.w_g32 = (const float *)c->wg32.p;
    a.wgt32 = (const float *)c->wgt32.p;
    a.cn = (const unsigned long long *)c->cn.p;
    a.cg = (const unsigned long long *)c->cg.p;
    a.counts_in_smem = mcrt::fp32_plain_stage_fits(c->nb, c->ng) ? 1 : 0;
    a.guide = (const unsigned short *)c->guide.p;
    a.gguide = (const unsigned char *)c->gguide.p;
    if (p->proposal == MCRT_PROPOSAL_CELL) {
      a.cell_cn = (const unsigned long long *)c->cell_cn.p;
      a.cell_cg = (const unsigned long long *)c->cell_cg.p;
      a.cell_hemi = (const unsigned int *)c->cell_hemi.p;
      if (mcrt::fp32_cell_stage_fits(c->nb, c->ng)) a.counts_in_smem |= 2;
    }
    a.rays = p->rays_per_cell;
    a.max_steps = p->max_steps;
    a.mg_levels = p->mg_levels > 1 ? p->mg_levels : 1;
    a.mg_steps = p->mg_levels > 1 ? p->mg_steps : 0x7fffffff;
    a.origin = p->origin;
    a.tol = p->tol;
    set_float_copies(&a);
    a.key0 = (unsigned)(p->seed & 0xffffffffu);
    a.key1 = (unsigned)(p->seed >> 32);
    set_round_keys(&a);
    a.claim_rays = items[0].ctx->claim_rays;
    a.snapshot = items[k].snapshot;
    a.ray_offset_dev = b->d_offset;
    a.bnx = g.nx;
    a.bny = g.ny;
    a.bnz = g.nz;
    a.ncells_box = (long long)g.nx * g.ny * g.nz;
    a.q = items[k].q_out;
    a.sigma = items[k].sigma_out;
    P[k] = mcrt::fp32_bricks_positions(a.bnx, a.bny, a.bnz);
    long long pc = ((long long)c->scratch_mib << 20) / ((long long)p->rays_per_cell * (long long)sizeof(float));
    if (pc < 1) pc = 1;
    if (pc > P[k]) pc = P[k];
    Pc[k] = pc;
    void *ct = nullptr;
    BK(cudaMalloc(&ct, mcrt::NCOUNTERS * sizeof(unsigned long long)), "alloc counters");
    b->owned.push_back(ct);
    a.counters = (unsigned long long *)ct;
    b->counters.push_back((unsigned long long *)ct);
    w[k] = weights ? weights[k] : (double)a.ncells_box;
    wsum += w[k];
  }
  mcrt_ctx *c0 = items[0].ctx;
  // Snapshots that share the k-distribution run as ONE persistent trace launch
  // (and one reduction) over all their cells: warps claim runs of brick-ordered
  // positions of the concatenated snapshots, largest snapshot first (unless
  // items[0]'s tuning asks for per-item launches).
  bool same_kdist = n <= mcrt::fp32_batch_max_snapshots() && !items[0].ctx->batch_per_snapshot;
  for (int k = 0; k < n && same_kdist; ++k)
    if (items[k].ctx->grid.xz_walls) same_kdist = false;  // closed boxes: per-snapshot kernels
  for (int k = 1; k < n && same_kdist; ++k) {
    const mcrt_ctx *c = items[k].ctx;
    same_kdist = c->nb == c0->nb && c->ng == c0->ng && c->nT == c0->nT && c->T0 == c0->T0 &&
                 c->dT == c0->dT && c->x_ref == c0->x_ref && c->w_g == c0->w_g &&
                 c->kappa == c0->kappa && c->B == c0->B;
  }
  if (same_kdist) {
    std::vector<int> order(n);
    for (int k = 0; k < n; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return P[x] > P[y]; });
    std::vector<mcrt::SnapArgs> sn(n + 1);
    std::memset(sn.data(), 0, sizeof(mcrt::SnapArgs) * (n + 1));
    long long pos = 0;
    for (int r = 0; r < n; ++r) {
      const int k = order[r];
      const mcrt::TraceArgs &a = args[k];
      mcrt::SnapArgs &t = sn[r];
      t.fpos32 = a.fpos32;
      t.yf32 = a.yf32;
      t.bwall32 = a.bwall32;
      t.wgt32 = a.wgt32;
      t.cn = a.cn;
      t.cg = a.cg;
      t.guide = a.guide;
      t.cell_cn = a.cell_cn;
      t.cell_cg = a.cell_cg;
      t.cell_hemi = a.cell_hemi;
      t.q = a.q;
      t.sigma = a.sigma;
      t.p0 = pos;
      t.nx = a.nx;
      t.ny = a.ny;
      t.nz = a.nz;
      t.reflect = a.reflect;
      t.dx = (float)a.dx;
      t.dy = (float)a.dy;
      t.dz = (float)a.dz;
      t.eps0 = (float)a.eps_wall[0];
      t.eps1 = (float)a.eps_wall[1];
      t.snapshot = a.snapshot;
      pos += P[k];
    }
    sn[n].p0 = pos;
    void *d_sn = nullptr;
    BK(cudaMalloc(&d_sn, sizeof(mcrt::SnapArgs) * (n + 1)), "alloc snapshots");
    b->owned.push_back(d_sn);
    BK(cudaMemcpy(d_sn, sn.data(), sizeof(mcrt::SnapArgs) * (n + 1), cudaMemcpyHostToDevice), "copy snapshots");
    // sample scratch: the whole batch when at most half the free memory, else chunks
    size_t fr = 0, tot = 0;
    BK(cudaMemGetInfo(&fr, &tot), "memory info");
    const size_t per_pos = (size_t)p->rays_per_cell * sizeof(float);
    long long pc = (long long)((fr / 2) / per_pos);
    if (pc < 1) pc = 1;
    if (pc > pos) pc = pos;
    void *yb = nullptr, *ct = nullptr;
    BK(cudaMalloc(&yb, (size_t)pc * per_pos), "alloc sample scratch");
    b->owned.push_back(yb);
    BK(cudaMalloc(&ct, mcrt::NCOUNTERS * sizeof(unsigned long long)), "alloc counters");
    b->owned.push_back(ct);
    b->counters.assign(1, (unsigned long long *)ct);
    mcrt::TraceArgs a = args[order[0]];
    a.snaps = (const mcrt::SnapArgs *)d_sn;
    a.nsnaps = n;
    a.batch_stretched = 0;
    for (int k = 0; k < n; ++k)
      if (args[k].yf32) a.batch_stretched = 1;
    a.ybuf = (float *)yb;
    a.step_acc = nullptr;
    a.steps_cell = nullptr;
    a.ray_steps = nullptr;
    a.counters = (unsigned long long *)ct;
    a.grid_blocks = 0;
    a.long_rays = nullptr;
    a.long_cap = 0;
    a.long_steps = c0->long_steps > 0 ? c0->long_steps : 0x7fffffff;
    a.long_flight = c0->long_flight;
    if (c0->long_steps > 0 && a.mg_levels <= 1) {
      const long long lc = mcrt::long_ray_capacity(pc * (long long)p->rays_per_cell, c0->long_steps);
      void *lb = nullptr;
      BK(cudaMalloc(&lb, (size_t)lc * sizeof(mcrt::LongRay)), "alloc long-ray buffer");
      b->owned.push_back(lb);
      a.long_rays = (mcrt::LongRay *)lb;
      a.long_cap = (int)lc;
    }
    int bps = 0, nsm = 0;
    BK(mcrt::prepare_trace_fp32_batch(c0->min_blocks, c0->steps_per_round, a.nb, a.ng, n, a.counts_in_smem,
                                      a.mg_levels > 1, &bps, &nsm),
       "prepare launch");
    b->streams.assign(1, nullptr);
    BK(cudaStreamCreateWithFlags(&b->streams[0], cudaStreamNonBlocking), "stream");
    BK(cudaDeviceSynchronize(), "sync");
    cudaStream_t s0 = b->streams[0];
    BK(cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal), "begin capture");
    cudaError_t ce = cudaMemsetAsync(a.counters, 0, mcrt::NCOUNTERS * sizeof(unsigned long long), s0);
    int launches = 0;
    for (long long p0 = 0; p0 < pos && ce == cudaSuccess; p0 += pc) {
      a.chunk_p0 = p0;
      a.chunk_p1 = p0 + pc < pos ? p0 + pc : pos;
      ce = mcrt::launch_trace_fp32_batch(a, c0->min_blocks, c0->steps_per_round, s0);
      launches += mcrt::long_rays_on(a) ? 3 : 2;
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(s0, &graph);
    b->graph = graph;
    if (ce != cudaSuccess) return bail(MCRT_E_CUDA, ce, "capture");
    if (ee != cudaSuccess) return bail(MCRT_E_CUDA, ee, "end capture");
    BK(cudaGraphInstantiate(&b->exec, b->graph, 0), "instantiate graph");
    b->launches = launches;
    b->single_launch = true;
    *out = b;
    return MCRT_OK;
  }
  // Otherwise one graph of per-snapshot launches.  Persistent CTAs: with
  // weights, one wave shared by the items in proportion to their work (all
  // items run at once); without, each item's kernel is a full wave and `streams`
  // branches run items in decreasing order of work, so one kernel's tail
  // overlaps the next kernel's start.
  int bps = 0, nsm = 0;
  BK(mcrt::prepare_trace_fp32(c0->min_blocks, c0->steps_per_round, args[0].nb, args[0].ng,
                              args[0].counts_in_smem, args[0].mg_levels > 1, &bps, &nsm),
     "prepare launch");
  const long long total = (long long)bps * nsm;
  std::vector<int> order(n);
  for (int k = 0; k < n; ++k) order[k] = k;
  std::sort(order.begin(), order.end(), [&](int x, int y) { return w[x] > w[y]; });
  b->streams.assign(streams, nullptr);
  b->joins.assign(streams, nullptr);
  for (int k = 0; k < streams; ++k) {
    BK(cudaStreamCreateWithFlags(&b->streams[k], cudaStreamNonBlocking), "stream");
    BK(cudaEventCreateWithFlags(&b->joins[k], cudaEventDisableTiming), "event");
  }
  for (int k = 0; k < n; ++k) {
    long long blocks = weights ? (long long)((double)total * w[k] / wsum + 0.5) : total;
    args[k].grid_blocks = (int)(blocks < 1 ? 1 : blocks);
  }
  // items of one branch run one after another, so they share its scratch
  for (int j = 0; j < streams; ++j) {
    long long pmax = 0;
    for (int r = j; r < n; r += streams) pmax = Pc[order[r]] > pmax ? Pc[order[r]] : pmax;
    void *yb = nullptr, *sa = nullptr, *lb = nullptr;
    BK(cudaMalloc(&yb, (size_t)pmax * p->rays_per_cell * sizeof(float)), "alloc sample scratch");
    b->owned.push_back(yb);
    BK(cudaMalloc(&sa, (size_t)pmax * sizeof(unsigned long long)), "alloc step scratch");
    b->owned.push_back(sa);
    const long long lc = mcrt::long_ray_capacity(pmax * (long long)p->rays_per_cell, c0->long_steps);
    if (c0->long_steps > 0) {
      BK(cudaMalloc(&lb, (size_t)lc * sizeof(mcrt::LongRay)), "alloc long-ray buffer");
      b->owned.push_back(lb);
    }
    for (int r = j; r < n; r += streams) {
      mcrt::TraceArgs &ak = args[order[r]];
      ak.ybuf = (float *)yb;
      ak.step_acc = (unsigned long long *)sa;
      ak.long_rays = (mcrt::LongRay *)lb;
      ak.long_cap = lb ? (int)lc : 0;
      ak.long_steps = c0->long_steps > 0 ? c0->long_steps : 0x7fffffff;
      ak.long_flight = c0->long_flight;
    }
  }
  BK(cudaDeviceSynchronize(), "sync");
  // capture: fork -> branch j runs its items [clear counters, chunks of trace (+ long rays) + reduce] -> join
  cudaStream_t s0 = b->streams[0];
  BK(cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal), "begin capture");
  cudaError_t ce = cudaEventRecord(b->fork, s0);
  for (int j = 1; j < streams && ce == cudaSuccess; ++j) ce = cudaStreamWaitEvent(b->streams[j], b->fork, 0);
  int launches = 0;
  for (int r = 0; r < n && ce == cudaSuccess; ++r) {
    const int k = order[r];
    cudaStream_t sk = b->streams[r % streams];
    ce = cudaMemsetAsync(args[k].counters, 0, mcrt::NCOUNTERS * sizeof(unsigned long long), sk);
    for (long long p0 = 0; p0 < P[k] && ce == cudaSuccess; p0 += Pc[k]) {
      args[k].chunk_p0 = p0;
      args[k].chunk_p1 = p0 + Pc[k] < P[k] ? p0 + Pc[k] : P[k];
      int kn = 0;
      ce = mcrt::launch_trace_fp32(args[k], c0->min_blocks, c0->steps_per_round, sk, nullptr, &kn);
      launches += kn;
    }
  }
  for (int j = 1; j < streams && ce == cudaSuccess; ++j) {
    ce = cudaEventRecord(b->joins[j], b->streams[j]);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(s0, b->joins[j], 0);
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(s0, &graph);
  b->graph = graph;
  if (ce != cudaSuccess) return bail(MCRT_E_CUDA, ce, "capture");
  if (ee != cudaSuccess) return bail(MCRT_E_CUDA, ee, "end capture");
  BK(cudaGraphInstantiate(&b->exec, b->graph, 0), "instantiate graph");
  b->launches = launches;
#undef BK
  *out = b;
  return MCRT_OK;
}

extern "C" int mcrt_batch_run(mcrt_batch *b, uint64_t ray_offset, void *stream) {
  if (!b) return MCRT_E_ARG;
  if ((unsigned long long)ray_offset + (unsigned long long)b->rays > (1ull << 32))
    return batch_fail(b, MCRT_E_ARG, "ray indices beyond 2^32");
  DeviceGuard dg(b->device);
  if (!dg.ok) return batch_fail(b, MCRT_E_CUDA, "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  b->h_offset = ray_offset;  // pageable source: staged before cudaMemcpyAsync returns
  cudaError_t e = cudaMemcpyAsync(b->d_offset, &b->h_offset, sizeof(b->h_offset),
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaEventRecord(b->ev0, s);
  if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, s);
  if (e == cudaSuccess) e = cudaEventRecord(b->ev1, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return batch_fail(b, MCRT_E_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
  }
  b->ran = true;
  b->last_stream = s;
  return MCRT_OK;
}

extern "C" int mcrt_batch_get_stats(mcrt_batch *b, mcrt_solve_stats *out) {
  if (!b || !out) return MCRT_E_ARG;
  if (!b->ran) return batch_fail(b, MCRT_E_STATE, "no run yet");
  DeviceGuard dg(b->device);
  if (!dg.ok) return batch_fail(b, MCRT_E_CUDA, "cudaSetDevice");
  std::memset(out, 0, sizeof(*out));
  cudaError_t e = cudaEventSynchronize(b->ev1);
  for (unsigned long long *cp : b->counters) {
    unsigned long long cnt[mcrt::NCOUNTERS];
    if (e == cudaSuccess) e = cudaMemcpy(cnt, cp, sizeof(cnt), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) break;
    if (cnt[5] != 0) return batch_fail(b, MCRT_E_TIMEOUT, "trace kernel stopped without progress");
    out->steps += cnt[0];
    out->capped += cnt[1];
    out->wall_hits += cnt[2];
    out->rays += cnt[3];
    if (cnt[4] > out->max_ray_steps) out->max_ray_steps = cnt[4];
    out->long_rays += cnt[8];
    out->long_overflow += cnt[9];
  }
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, b->ev0, b->ev1);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return batch_fail(b, MCRT_E_CUDA, std::string("batch stats: ") + cudaGetErrorString(e));
  }
  out->kernel_ms = ms;
  out->launches = b->launches;
  return MCRT_OK;
}

extern "C" const char *mcrt_batch_last_error(const mcrt_batch *b) { return b ? b->err.c_str() : ""; }

extern "C" int mcrt_batch_destroy(mcrt_batch *b) {
  if (!b) return MCRT_OK;
  {
    DeviceGuard dg(b->device);
    if (b->ran && b->ev1) cudaEventSynchronize(b->ev1);
    batch_release(b);
  }
  delete b;
  return MCRT_OK;
}
